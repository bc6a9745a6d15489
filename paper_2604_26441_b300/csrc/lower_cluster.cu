// The bottom of the V-cycle (Eq. vcycle) -- the last assembled level m and the
// coarsest solve -- in one launch of one thread-block cluster.
//
// At 100^3 level m has 2,197 nodes and the coarsest level 882 free DOFs.  As
// separate launches, each of the ~10 steps there (restriction and first
// smoothing step, smoothing steps, residual, restriction, coarsest solve,
// prolongation, smoothing steps) costs a launch and a few dependent memory
// round trips on an idle GPU.  Here a cluster of CTAs keeps level m's operator
// in shared memory and separates the steps with the cluster's hardware
// barrier (barrier.cluster arrive.release / wait.acquire), which orders the
// global writes of one step before the reads of the next across the cluster.
//
// Layout: CTA k owns the level-m nodes [k R, (k+1) R) (R = ceil(nn / CTAs)).
// It holds their rows of the operator expanded to all 27 neighbour blocks (the
// backward blocks transposed from the neighbours' forward blocks of the
// symmetric-half storage), their right-hand side, Jacobi scale, Chebyshev
// increment and masks.  Before each operator application every CTA copies the
// whole current level-m vector into shared memory, so all of a row's operands
// are local; a thread forms one output component (81 products, two partial
// sums).  The steps' arithmetic (coefficient tables, masks, the trilinear
// transfers with the odd-size clamp) is that of the per-level kernels; the sum
// order of the operator rows differs, so results agree to rounding.
//
// Opt-in (gmg_options.lower_cluster): at 100^3 the one launch took 59 us on its
// 16 SMs against ~40 us for the per-level launches on the whole GPU.
//
// The coarsest solve applies the Cholesky-derived inverse in double-float:
// Ainv = Ahi + Alo (FP32 parts of the FP64 inverse), each product split exactly
// with an FMA and a row summed in double-float on the FP32 pipes (~44
// significant bits; the result is FP32).  On the cluster's few SMs an FP64
// GEMV would be bound by the FP64 pipe.
#include <algorithm>
#include <cooperative_groups.h>

#include "internal.cuh"

namespace gmg {

namespace {

namespace cg = cooperative_groups;

constexpr int kLcThreads = 1024;
constexpr int kLcCtas = 16;  // cluster size (non-portable: needs the opt-in attribute)

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

// shared-memory layout of one CTA (offsets in bytes, each 16-byte aligned)
struct LcLayout {
    int R;        // rows (owned nodes) per CTA
    int nn;       // level-m nodes
    int nL;       // coarsest free DOFs
    size_t a_off, x_off, b_off, inv_off, d_off, msk_off, bc_off, bytes;
};
__host__ __device__ inline size_t lc_al16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline LcLayout lc_layout(int nn, int nL) {
    LcLayout L{};
    L.nn = nn;
    L.nL = nL;
    L.R = (nn + kLcCtas - 1) / kLcCtas;
    size_t o = 0;
    L.a_off = o;   o = lc_al16(o + sizeof(float) * 243 * (size_t)L.R);
    L.x_off = o;   o = lc_al16(o + sizeof(float) * 3 * (size_t)nn);
    L.b_off = o;   o = lc_al16(o + sizeof(float) * 3 * (size_t)L.R);
    L.inv_off = o; o = lc_al16(o + sizeof(float) * 3 * (size_t)L.R);
    L.d_off = o;   o = lc_al16(o + sizeof(float) * 3 * (size_t)L.R);
    L.msk_off = o; o = lc_al16(o + (size_t)L.R);
    L.bc_off = o;  o = lc_al16(o + sizeof(float) * (size_t)(nL > 1 ? nL : 1));
    L.bytes = o;
    return L;
}

}  // namespace



namespace {

// 1D restriction weights (Eq. trilinear_weights, odd-size clamp): coarse node I
// takes fine nodes idx[0..2] with weights w[0..2] (0 where a node does not exist)
__device__ __forceinline__ void lc_support3(int I, int nf, int idx[3], float w[3]) {
    const int nc = nf >> 1, f = 2 * I + 1;
    idx[0] = I >= 1 ? 2 * I - 1 : 2 * I; w[0] = I >= 1 ? 0.5f : 0.f;
    idx[1] = 2 * I; w[1] = 1.f;
    idx[2] = f <= nf ? f : 2 * I; w[2] = f <= nf ? (f < 2 * nc ? 0.5f : 1.f) : 0.f;
}
// 1D prolongation parents of fine node f
__device__ __forceinline__ void lc_parents2(int f, int nf, int idx[2], float w[2]) {
    const int nc = nf >> 1;
    if ((f & 1) == 0) { idx[0] = idx[1] = f >> 1; w[0] = 1.f; w[1] = 0.f; }
    else if (f < 2 * nc) { idx[0] = (f - 1) >> 1; idx[1] = (f + 1) >> 1; w[0] = w[1] = 0.5f; }
    else { idx[0] = idx[1] = nc; w[0] = 1.f; w[1] = 0.f; }
}
// (P^T t)[n] (unmasked) for coarse node n of a level with cnx x cny nodes per
// plane minus one; t a dense vector of the finer level (fnx, fny, fnz).  The
// same products and order as the per-node restriction kernels.
__device__ __forceinline__ void lc_restrict(int n, int CX, int CY, int fnx, int fny, int fnz, const float* t,
                                            float out[3]) {
    const int FX = fnx + 1, FY = fny + 1;
    const int I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    lc_support3(I, fnx, ix, wx);
    lc_support3(J, fny, iy, wy);
    lc_support3(K, fnz, iz, wz);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float w = wx[a] * wy[b] * wz[c];
                const int f = ix[a] + FX * (iy[b] + FY * iz[c]);
                s0 = fmaf(w, __ldcg(t + 3 * f), s0);
                s1 = fmaf(w, __ldcg(t + 3 * f + 1), s1);
                s2 = fmaf(w, __ldcg(t + 3 * f + 2), s2);
            }
    out[0] = s0; out[1] = s1; out[2] = s2;
}

__global__ void __launch_bounds__(kLcThreads, 1) k_lower_cluster(LowerClusterArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const CoarseLevel& M = a.m;
    const LcLayout lay = lc_layout(M.nn, a.nL);
    float* As = reinterpret_cast<float*>(sm + lay.a_off);     // [R][27 slots][3 x 3]
    float* xs = reinterpret_cast<float*>(sm + lay.x_off);     // [nn][3], the current level-m vector
    float* bs = reinterpret_cast<float*>(sm + lay.b_off);     // [R][3] right-hand side
    float* ivs = reinterpret_cast<float*>(sm + lay.inv_off);  // [R][3] Jacobi scale
    float* ds = reinterpret_cast<float*>(sm + lay.d_off);     // [R][3] Chebyshev increment
    uint8_t* ms = sm + lay.msk_off;                           // [R] masks
    float* bcs = reinterpret_cast<float*>(sm + lay.bc_off);   // [nL] coarsest right-hand side (free DOFs)
    const int rank = (int)cl.block_rank(), tid = threadIdx.x;
    const int NX = M.nx + 1, NY = M.ny + 1, NZ = M.nz + 1, nn = M.nn, R = lay.R;
    const int n0 = rank * R, rows = max(0, min(n0 + R, nn) - n0);
    const long long N = M.ps;
    pdl_entry();

    // ---- this CTA's rows: the 27 neighbour blocks, Jacobi scale and masks
    for (int q = tid; q < rows * 27; q += kLcThreads) {
        const int r = q / 27, sl = q - 27 * r, n = n0 + r;
        const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
        const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
        const bool in = i + dx >= 0 && i + dx < NX && j + dy >= 0 && j + dy < NY && k + dz >= 0 && k + dz < NZ;
        float* E = As + 243 * r + 9 * sl;
        if (!in) {
#pragma unroll
            for (int e = 0; e < 9; ++e) E[e] = 0.f;
        } else if (sl >= 13) {  // diagonal and forward blocks, stored at n
            const float* A = M.A + (long long)(sl - 13) * 9 * N + n;
#pragma unroll
            for (int e = 0; e < 9; ++e) E[e] = __ldg(A + e * N);
        } else {  // backward: the transpose of the neighbour's forward block toward n
            const int nb = n + dx + NX * (dy + NY * dz);
            const float* A = M.A + (long long)(13 - sl) * 9 * N + nb;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int ci = 0; ci < 3; ++ci) E[3 * c + ci] = __ldg(A + (3 * ci + c) * N);
        }
    }
    for (int q = tid; q < rows * 3; q += kLcThreads) ivs[q] = __ldg(M.invdiag + 3 * (long long)n0 + q);
    for (int r = tid; r < rows; r += kLcThreads) ms[r] = __ldg(M.mask + n0 + r);

    // y[c] of own row r from the staged vector xs (81 products, two partial sums)
    auto row_apply = [&](int r, int c) -> float {
        const int n = n0 + r;
        const float* E = As + 243 * r + 3 * c;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int sl = 0; sl < 27; ++sl) {
            const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
            int nb = n + dx + NX * (dy + NY * dz);
            nb = nb < 0 ? 0 : (nb >= nn ? nn - 1 : nb);  // out-of-grid blocks are zero
            const float* xv = xs + 3 * nb;
            const float t = fmaf(E[9 * sl + 2], xv[2], fmaf(E[9 * sl + 1], xv[1], E[9 * sl] * xv[0]));
            if (sl & 1) s1 += t;
            else s0 += t;
        }
        return s0 + s1;
    };
    // the whole current vector into shared memory (written by all CTAs before the barrier)
    auto stage_x = [&](const float* x) {
        const int n4 = (3 * nn) / 4;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        float4* s4 = reinterpret_cast<float4*>(xs);
        for (int q = tid; q < n4; q += kLcThreads) s4[q] = __ldcg(x4 + q);
        for (int q = 4 * n4 + tid; q < 3 * nn; q += kLcThreads) xs[q] = __ldcg(x + q);
        __syncthreads();
    };
    float* const buf[2] = {M.x2, M.x};  // the per-level path's write order: S, X, S, ...
    int writes = 0;
    const bool cheb = M.kind == GMG_SMOOTHER_CHEBYSHEV;
    // one smoothing step (k > 0 or post-smoothing) from the staged vector
    auto smooth = [&](int k, bool write_d) {
        const float cd = (float)M.coef[2 * k], ca = (float)M.coef[2 * k + 1];
        float* out = buf[writes & 1];
        for (int q = tid; q < rows * 3; q += kLcThreads) {
            const int r = q / 3, c = q - 3 * r, n = n0 + r;
            const float y = row_apply(r, c);
            float xn = 0.f, dn = 0.f;
            if (!fixed_bit(ms[r], c)) {
                dn = ca * ivs[q] * (bs[q] - y);
                if (cd != 0.f) dn = fmaf(cd, ds[q], dn);
                xn = xs[3 * n + c] + dn;
            }
            out[3 * n + c] = xn;
            if (write_d) ds[q] = dn;
        }
        ++writes;
    };

    // ---- pre-smoothing: the restriction of the finer residual into b and the
    // first step from a zero iterate (x = c_a D^-1 b, d = x), then steps 1..
    {
        const float ca = (float)M.coef[1];
        float* out = buf[writes & 1];
        for (int r = tid; r < rows; r += kLcThreads) {
            const int n = n0 + r;
            float bc[3];
            lc_restrict(n, NX, NY, a.fnx, a.fny, a.fnz, a.ft, bc);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int q = 3 * r + c;
                const float bv = fixed_bit(ms[r], c) ? 0.f : bc[c];
                bs[q] = bv;
                M.b[3 * n + c] = bv;  // read again by a second visit of the level (W-cycle)
                const float v = ca * ivs[q] * bv;  // the scale is 0 on fixed DOFs
                out[3 * n + c] = v;
                if (cheb && M.degree > 1) ds[q] = v;
            }
        }
        ++writes;
    }
    for (int k = 1; k < M.degree; ++k) {
        cl.sync();
        stage_x(buf[(writes - 1) & 1]);
        smooth(k, cheb && k != M.degree - 1);
    }
    // ---- residual t = b - K x of the pre-smoothed iterate
    float* const cur = buf[(writes - 1) & 1];
    cl.sync();
    stage_x(cur);
    for (int q = tid; q < rows * 3; q += kLcThreads) {
        const int r = q / 3, c = q - 3 * r;
        const float y = row_apply(r, c);
        M.t[3 * (n0 + r) + c] = fixed_bit(ms[r], c) ? 0.f : bs[q] - y;
    }
    cl.sync();
    // ---- restriction of t into the coarsest level, over the whole cluster
    const int gt = rank * kLcThreads + tid, gstride = kLcCtas * kLcThreads;
    for (int n = gt; n < a.cnn; n += gstride) {
        float bc[3];
        lc_restrict(n, a.cnx + 1, a.cny + 1, M.nx, M.ny, M.nz, M.t, bc);
        const uint8_t m = a.cmask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) a.cb[3 * n + c] = fixed_bit(m, c) ? 0.f : bc[c];
    }
    cl.sync();
    // ---- coarsest solve: x = (Ahi + Alo) b on the free DOFs, 0 on the fixed ones
    for (int q = gt; q < 3 * a.cnn; q += gstride)
        if (fixed_bit(a.cmask[q / 3], q % 3)) a.cx[q] = 0.f;
    for (int j = tid; j < a.nL; j += kLcThreads) bcs[j] = __ldcg(a.cb + a.free_idx[j]);
    __syncthreads();
    {
        const int lane = tid & 31, gw = rank * (kLcThreads / 32) + (tid >> 5), nw = kLcCtas * (kLcThreads / 32);
        for (int row = gw; row < a.nL; row += nw) {
            const float* ah = a.Ahi + (long long)row * a.nL;
            const float* al = a.Alo + (long long)row * a.nL;
            float hi = 0.f, lo = 0.f;
            for (int j = lane; j < a.nL; j += 32) {
                const float av = __ldg(ah + j), av2 = __ldg(al + j), bv = bcs[j];
                const float pr = __fmul_rn(av, bv);
                const float e = __fmaf_rn(av, bv, -pr);
                const float sm2 = __fadd_rn(hi, pr);
                const float bb = __fsub_rn(sm2, hi);
                const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm2, bb)), __fsub_rn(pr, bb));
                hi = sm2;
                lo = __fadd_rn(lo, __fadd_rn(t, __fmaf_rn(av2, bv, e)));
            }
            double sv = f2d_exact(hi) + f2d_exact(lo);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sv += __shfl_down_sync(0xffffffffu, sv, o);
            if (lane == 0) a.cx[a.free_idx[row]] = (float)sv;
        }
    }
    cl.sync();
    // ---- prolongation: cur += P x_coarse on the free DOFs of the own nodes
    for (int r = tid; r < rows; r += kLcThreads) {
        const int n = n0 + r;
        const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
        const int CX = a.cnx + 1, CY = a.cny + 1;
        int ix[2], iy[2], iz[2];
        float wx[2], wy[2], wz[2];
        lc_parents2(i, M.nx, ix, wx);
        lc_parents2(j, M.ny, iy, wy);
        lc_parents2(k, M.nz, iz, wz);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float w = wx[q] * wy[b] * wz[c];
                    const int m = ix[q] + CX * (iy[b] + CY * iz[c]);
                    s0 = fmaf(w, __ldcg(a.cx + 3 * m), s0);
                    s1 = fmaf(w, __ldcg(a.cx + 3 * m + 1), s1);
                    s2 = fmaf(w, __ldcg(a.cx + 3 * m + 2), s2);
                }
        const float sv[3] = {s0, s1, s2};
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (!fixed_bit(ms[r], c)) cur[3 * n + c] = __ldcg(cur + 3 * n + c) + sv[c];
    }
    // ---- post-smoothing from the corrected iterate
    for (int k = 0; k < M.degree; ++k) {
        cl.sync();
        stage_x(buf[(writes - 1) & 1]);
        smooth(k, cheb && k != M.degree - 1);
    }
}

}  // namespace

// Shared memory of the cluster path for a last assembled level of nn nodes and
// nL coarsest free DOFs (bytes per CTA).
size_t lower_cluster_smem(int nn, int nL) { return lc_layout(nn, nL).bytes; }

// Whether one cluster of kLcCtas CTAs with that shared memory can be resident;
// sets the kernel's attributes once.
bool lower_cluster_available(size_t smem) {
    if (smem > 220 * 1024) return false;
    if (cudaFuncSetAttribute(k_lower_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_lower_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kLcCtas);
    cfg.blockDim = dim3(kLcThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLcCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_lower_cluster, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters >= 1;
}

void launch_lower_cluster(const LowerClusterArgs& a, size_t smem, cudaStream_t s) {
    note_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kLcCtas);
    cfg.blockDim = dim3(kLcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLcCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, k_lower_cluster, a);
}


namespace {
// hi = (float)A, lo = (float)(A - hi): the FP32 parts of the coarsest inverse
__global__ void k_lc_split(const double* A, long long n, float* hi, float* lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = A[i];
        const float h = (float)v;
        hi[i] = h;
        lo[i] = (float)(v - (double)h);
    }
}
}  // namespace

void launch_split_inverse(const double* A, long long n, float* hi, float* lo, cudaStream_t s) {
    note_launch();
    k_lc_split<<<148 * 4, 256, 0, s>>>(A, n, hi, lo);
}

}  // namespace gmg
