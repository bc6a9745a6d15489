// FP64 true residual of the fine level, r = f - K u, with ||r_free||^2 per block
// (Sec. "Outer Krylov Solver and Convergence Statement": solves are accepted
// only by the true residual, computed here in FP64 from the FP64 moduli and the
// FP64 iterate).
//
// Same factorisation and schedule as the FP32 fine operator (fine.cu): K_e =
// H^T G H with G in eight 3x3 parity-class blocks, one thread per element column
// marching along z, face difference sums shared between layers, and the node
// sums formed by warp shuffles and a shared-memory exchange.
//
// Arithmetic.  FP64 runs at about 1/64 of the FP32 rate on this part, and the
// ~200 FP64 operations per element of the factored form kept the FP64 pipe 82 %
// busy for 0.56 ms at 100^3.  The element arithmetic therefore runs in
// double-float form instead: a value is an unevaluated sum hi + lo of two FP32
// numbers (~44 significant bits), added with Knuth's error-free TwoSum and
// multiplied with an FMA-based exact product (Dekker's scheme), followed by a
// renormalisation.  Each double-float operation costs ~6-10 FP32 instructions
// and its error stays within a few units of 2^-44 of its operands' magnitude,
// far below what a 1e-6 acceptance test needs (the result agrees with a plain
// FP64 evaluation to ~1e-13).  FP64 remains for what is read and written: u,
// f and E are FP64 and split once per value; f - K u, r and ||r||^2 are
// formed in FP64.
#include <algorithm>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int BX = 16, BY = 16, NT = BX * BY;

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

// ---- double-float numbers: value = hi + lo, |lo| <= ulp(hi) / 2 ----------------
// The intrinsics (__fadd_rn, __fmul_rn) are never contracted into FMAs, which
// the error-free transformations rely on.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df df_of(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }
// TwoSum of the high parts, the low parts added to its error, renormalised.
__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// Exact product of the high parts by an FMA, cross terms added, renormalised.
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
// lane arithmetic of the symmetric contraction (gsym_contract) in double-float
__device__ __forceinline__ df g_add(df a, df b) { return a + b; }
__device__ __forceinline__ df g_mul(df a, df b) { return a * b; }
__device__ __forceinline__ df g_fma(df a, df b, df c) { return a * b + c; }
__device__ __forceinline__ df shfl_down(df a, int d, int w) {
    return {__shfl_down_sync(0xffffffffu, a.hi, d, w), __shfl_down_sync(0xffffffffu, a.lo, d, w)};
}

// The eight values of G's symmetric form (GSym order) as double-float pairs
// (split on the host from FP64).
struct GSymDF {
    float hi[8], lo[8];
};
GSymDF gsym_df(const double* g8) {
    GSymDF d;
    for (int k = 0; k < 8; ++k) {
        d.hi[k] = (float)g8[k];
        d.lo[k] = (float)(g8[k] - (double)d.hi[k]);
    }
    return d;
}

__device__ __forceinline__ void face_diffs(df u00, df u10, df u01, df u11, df q[4]) {
    const df dx0 = u10 - u00, dx1 = u11 - u01;
    q[1] = dx0 + dx1;
    q[2] = (u01 - u00) + (u11 - u10);
    q[3] = dx1 - dx0;
}

// Operands of one launch: one load (single-load calls), or up to kLoads loads
// whose blocks share the grid's z dimension (gz chunks per load).
struct ResidLoads {
    const double* f[kLoads];
    const double* u[kLoads];
    int gz;
    int pstride;  // partial sums of load l at partial[l * pstride ...]
};

__global__ void __launch_bounds__(NT, 1) k_resid64(int nx, int ny, int nz, const double* E, const uint8_t* mask,
                                                   const __grid_constant__ ResidLoads L, double* r64, float* r32,
                                                   int px, const double* sc, double* partial, GSymDF G, int zchunk) {
    pdl_entry();
    // load l of a multi-load launch: grid.z = L.gz chunks x loads, its own
    // f, u, scalar block and partial range
    const int l = (int)(blockIdx.z / (unsigned)L.gz), bz = (int)(blockIdx.z % (unsigned)L.gz);
    const double* f = L.f[l];
    const double* uvec = L.u[l];
    sc += l * SC_COUNT;
    partial += (long long)l * L.pstride;
    __shared__ df sp[2][BY + 1][(BX + 1) * 3];
    __shared__ df sx[2][BY][BX * 3];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1, NXY = NX * NY, NEXY = nx * ny;
    const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = bz * zchunk, k1 = min(k0 + zchunk, NZ);
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty, ox = cx + 1, oy = cy + 1;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const bool cell_in = cx >= 0 && cx < nx && cy >= 0 && cy < ny;
    const bool own_xy = cx >= 0 && cx < NX && cy >= 0 && cy < NY;
    const int own_base = cy * NX + cx, onode_base = oy * NX + ox, e_base = cy * nx + cx;
    const bool uzero = sc[SC_UNZ] == 0.0;  // u is identically zero: r = f

    int hx = 0, hy = 0;
    const bool halo = tid <= BX + BY;
    if (tid <= BX) { hx = tid; hy = BY; }
    else if (halo) { hx = BX; hy = tid - BX - 1; }
    const int hpx = x0 - 1 + hx, hpy = y0 - 1 + hy;
    const bool halo_xy = halo && hpx >= 0 && hpx < NX && hpy >= 0 && hpy < NY;
    const int halo_base = hpy * NX + hpx;

    double pv[3], ph[3];
    uint8_t pm = 7, phm = 7;
    auto prefetch = [&](int pz) {
        const bool zok = !uzero && pz >= 0 && pz < NZ;
        pv[0] = pv[1] = pv[2] = ph[0] = ph[1] = ph[2] = 0.0;
        pm = phm = 7;
        if (zok && own_xy) {
            const int n = own_base + pz * NXY;
            pv[0] = uvec[3 * n]; pv[1] = uvec[3 * n + 1]; pv[2] = uvec[3 * n + 2];
            pm = mask[n];
        }
        if (zok && halo_xy) {
            const int n = halo_base + pz * NXY;
            ph[0] = uvec[3 * n]; ph[1] = uvec[3 * n + 1]; ph[2] = uvec[3 * n + 2];
            phm = mask[n];
        }
    };
    auto store_plane = [&](int buf) {
        df* d = &sp[buf][ty][3 * tx];
        d[0] = df_of((pm & 1) ? 0.0 : pv[0]);
        d[1] = df_of((pm & 2) ? 0.0 : pv[1]);
        d[2] = df_of((pm & 4) ? 0.0 : pv[2]);
        if (halo) {
            df* e = &sp[buf][hy][3 * hx];
            e[0] = df_of((phm & 1) ? 0.0 : ph[0]);
            e[1] = df_of((phm & 2) ? 0.0 : ph[1]);
            e[2] = df_of((phm & 4) ? 0.0 : ph[2]);
        }
    };

    prefetch(k0 - 1);
    store_plane((k0 - 1) & 1);
    prefetch(k0);
    __syncthreads();
    const df zero{0.f, 0.f};
    df Qb[4][3], Cb[4][3], Tprev[4][3];
    for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 3; ++c) Qb[q][c] = Cb[q][c] = Tprev[q][c] = zero;
    {
        const int b = (k0 - 1) & 1;
        for (int c = 0; c < 3; ++c) {
            Cb[0][c] = sp[b][ty][3 * tx + c];
            Cb[1][c] = sp[b][ty][3 * (tx + 1) + c];
            Cb[2][c] = sp[b][ty + 1][3 * tx + c];
            Cb[3][c] = sp[b][ty + 1][3 * (tx + 1) + c];
            df q[4];
            face_diffs(Cb[0][c], Cb[1][c], Cb[2][c], Cb[3][c], q);
            for (int i = 1; i < 4; ++i) Qb[i][c] = q[i];
        }
    }
    double Enext = (!uzero && cell_in && k0 - 1 >= 0 && k0 - 1 < nz) ? E[e_base + (k0 - 1) * NEXY] : 0.0;
    bool pending = false;
    int pend_k = 0;
    df R1[3] = {zero, zero, zero};
    double rr = 0.0;

    auto finish = [&]() {
        const df* r0 = &sx[pend_k & 1][ty + 1][3 * tx];
        const int n = onode_base + pend_k * NXY;
        const uint8_t m = mask[n];
        for (int c = 0; c < 3; ++c) {
            const double v = fixed_bit(m, c) ? 0.0 : f[3 * n + c] - df_val(R1[c] + r0[c]);
            if (r64) r64[3 * n + c] = v;
            if (r32) r32[GMG_B(3 * (ox + px * (oy + NY * pend_k)) + c, 3LL * px * NY * NZ, 301)] = (float)v;
            rr += v * v;
        }
    };

    for (int kl = k0 - 1; kl < k1; ++kl) {
        const int pt = kl + 1;
        store_plane(pt & 1);
        __syncthreads();
        if (pending && owner) finish();
        pending = false;
        const df Ee = df_of(Enext);
        if (pt + 1 <= k1) prefetch(pt + 1);
        Enext = (!uzero && cell_in && kl + 1 < nz && kl + 1 < k1) ? E[e_base + (kl + 1) * NEXY] : 0.0;
        const int b = pt & 1;
        df Qt[4][3], Ct[4][3];
        for (int c = 0; c < 3; ++c) {
            Ct[0][c] = sp[b][ty][3 * tx + c];
            Ct[1][c] = sp[b][ty][3 * (tx + 1) + c];
            Ct[2][c] = sp[b][ty + 1][3 * tx + c];
            Ct[3][c] = sp[b][ty + 1][3 * (tx + 1) + c];
            df q[4];
            face_diffs(Ct[0][c], Ct[1][c], Ct[2][c], Ct[3][c], q);
            Qt[0][c] = zero;
            for (int i = 1; i < 4; ++i) Qt[i][c] = q[i];
        }
        df v[8][3];
        for (int c = 0; c < 3; ++c) {
            v[0][c] = zero;
            v[4][c] = ((Ct[0][c] - Cb[0][c]) + (Ct[1][c] - Cb[1][c])) + ((Ct[2][c] - Cb[2][c]) + (Ct[3][c] - Cb[3][c]));
            for (int q = 1; q < 4; ++q) {
                v[q][c] = Qt[q][c] + Qb[q][c];
                v[q + 4][c] = Qt[q][c] - Qb[q][c];
            }
        }
        df w[8][3];
        for (int c = 0; c < 3; ++c) w[0][c] = zero;
        {
            df g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) g[k] = Ee * df{G.hi[k], G.lo[k]};
            gsym_contract(GElem<df>{g[0], g[1], g[2], g[3], g[4], g[5], g[6], g[7]}, v, w);
        }
        df T[4][3], B[4][3];
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 3; ++c) {
                T[q][c] = w[q][c] + w[q + 4][c];
                B[q][c] = w[q][c] - w[q + 4][c];
            }
        if (kl >= k0) {
            df r0[3];
            for (int c = 0; c < 3; ++c) {
                const df S0 = Tprev[0][c] + B[0][c], S1 = Tprev[1][c] + B[1][c];
                const df S2 = Tprev[2][c] + B[2][c], S3 = Tprev[3][c] + B[3][c];
                const df p = S0 - S2, qd = S1 - S3, r = S0 + S2, sd = S1 + S3;
                const df c00 = p - qd, c10 = p + qd, c01 = r - sd, c11 = r + sd;
                R1[c] = c11 + shfl_down(c01, 1, BX);
                r0[c] = c10 + shfl_down(c00, 1, BX);
            }
            df* dst = &sx[kl & 1][ty][3 * tx];
            dst[0] = r0[0]; dst[1] = r0[1]; dst[2] = r0[2];
            pending = true;
            pend_k = kl;
        }
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 3; ++c) {
                Tprev[q][c] = T[q][c];
                Qb[q][c] = Qt[q][c];
                Cb[q][c] = Ct[q][c];
            }
    }
    __syncthreads();
    if (pending && owner) finish();
    // block sum of ||r||^2 in a fixed order
    __shared__ double wsum[NT / 32];
    for (int o = 16; o > 0; o >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, o);
    if ((tid & 31) == 0) wsum[tid >> 5] = rr;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < NT / 32; ++w2) s += wsum[w2];
        partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * bz)] = s;
    }
}

// Picks the z-chunk that minimises (waves x steps per block).  At ~230
// registers per thread one 256-thread block fits per SM, so a partial last wave
// costs a whole chunk of steps: at 100^3 (7 x 7 columns of blocks) chunks of 34
// planes give one wave of 147 blocks, where chunks of 15 gave 3 waves of 343.
dim3 resid_grid(int nx, int ny, int nz, int* zc_out, int nl = 1) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int gx = (NX + BX - 2) / (BX - 1), gy = (NY + BY - 2) / (BY - 1);
    static int slots = 0;
    if (slots == 0) {
        int dev = 0, sms = 148, per_sm = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid64, NT, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        slots = sms * per_sm;
    }
    int best_zc = NZ;
    long long best_cost = -1;
    for (int gz = 1; gz <= NZ; ++gz) {
        const int zc = (NZ + gz - 1) / gz;
        if (zc < 4 && gz > 1) break;
        const long long blocks = (long long)gx * gy * ((NZ + zc - 1) / zc) * nl;
        const long long cost = ((blocks + slots - 1) / slots) * (zc + 1);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_zc = zc;
        }
    }
    *zc_out = best_zc;
    return dim3(gx, gy, (NZ + best_zc - 1) / best_zc);
}

}  // namespace

int resid64_grid_blocks(int nx, int ny, int nz) {
    int zc = 0;
    const dim3 g = resid_grid(nx, ny, nz, &zc);
    return (int)(g.x * g.y * g.z);
}

void launch_fine_resid64(int nx, int ny, int nz, const double* E, const uint8_t* mask, const double* f, const double* u,
                         double* r64, float* r32, int px, const double* sc, double* partial, const double* g8,
                         cudaStream_t s) {
    int zc = 0;
    const dim3 g = resid_grid(nx, ny, nz, &zc);
    const GSymDF gd = gsym_df(g8);
    ResidLoads L{};
    L.f[0] = f;
    L.u[0] = u;
    L.gz = (int)g.z;
    note_launch();
    pdl_launch(k_resid64, dim3(g), dim3(dim3(BX, BY)), 0, s, nx, ny, nz, E, mask, L, r64, r32, px, sc, partial, gd,
               zc);
}

int resid64_grid_blocks_multi(int nx, int ny, int nz, int nl) {
    int zc = 0;
    const dim3 g = resid_grid(nx, ny, nz, &zc, nl);
    return (int)(g.x * g.y * g.z);
}

void launch_fine_resid64_multi(int nx, int ny, int nz, const double* E, const uint8_t* mask, int nl,
                               const double* const* f, const double* const* u, const double* sc, double* partial,
                               int pstride, const double* g8, cudaStream_t s) {
    int zc = 0;
    const dim3 g = resid_grid(nx, ny, nz, &zc, nl);
    const GSymDF gd = gsym_df(g8);
    ResidLoads L{};
    for (int l = 0; l < nl; ++l) {
        L.f[l] = f[l];
        L.u[l] = u[l];
    }
    L.gz = (int)g.z;
    L.pstride = pstride;
    note_launch();
    pdl_launch(k_resid64, dim3(g.x, g.y, g.z * nl), dim3(dim3(BX, BY)), 0, s, nx, ny, nz, E, mask, L,
               (double*)nullptr, (float*)nullptr, 0, sc, partial, gd, zc);
}

}  // namespace gmg
