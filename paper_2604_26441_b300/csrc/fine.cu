// Matrix-free fine-level operator (Eq. mf_matvec) fused with its consumers, for sm_103a.
//
// Formulation.  On the unit cube the 24x24 element stiffness K_e commutes with
// the reflections x -> 1-x, y -> 1-y, z -> 1-z.  In the basis of the eight
// monomials {1, X, Y, Z, XY, YZ, XZ, XYZ} of the corner signs (an 8-point
// Walsh-Hadamard transform H of the node values, per displacement component)
// it is block diagonal: the parity of (monomial, component) under the three
// reflections splits the 24 modes into 8 classes of 3, and
//     K_e = H^T G H,  G = H K_e H^T / 64,
// with G made of eight 3x3 blocks (72 numbers, 57 of them non-zero: the
// constant monomial is a rigid translation and drops out).  One element
// application costs 21 mode sums, 57 FMAs and 21 products with E_e instead of
// 576 FMAs, and every retained mode is a difference of nodal values, which keeps
// FP32 rounding proportional to the variation of u rather than its magnitude.
//
// Schedule.  A block of BX x BY threads (32x8 or 16x16, chosen per grid) owns a
// (BX-1) x (BY-1) patch of nodes and marches along z through a chunk of node
// planes; thread (tx, ty) holds the element column whose low corner is node
// (x0-1+tx, y0-1+ty).  Operands stream through shared-memory rings filled by
// cp.async (LDGSTS) several steps ahead: node planes and element moduli three
// layers ahead, smoother operands two planes ahead, so HBM latency is covered
// without register staging.  (TMA boxes do not fit here: a node row is 3(nx+1)
// floats, not a multiple of 16 bytes, so every row would be its own small box,
// and a TMA instruction takes warp-uniform operands, so the boxes of a step
// would issue one at a time.)  Per element layer a thread
//   - reads the four corner nodes of the layer's top plane from the ring,
//   - forms the x/y difference sums of the top plane once and reuses them for
//     the next layer (the Z mode is summed from per-corner z-differences),
//   - applies G and E_e, and converts the result back to face quantities,
//   - completes the node plane below: adds the top face of the previous layer,
//     expands to the four corners, sums the four cells around each node with a
//     warp shuffle (x) and a shared-memory exchange (y), and runs the epilogue
//     (apply / smoother step / residual) for its node one step later.
// The x and y components travel as packed f32x2 pairs, and the loop takes two
// layers per trip so that the layer state alternates between two register
// sets.  No atomics: every output is formed by its owner in a fixed order.
#include <algorithm>

#include "internal.cuh"

namespace gmg {

namespace {

// Monomial (bit 0 = X, 1 = Y, 2 = Z) of component c in parity class sigma.
__host__ __device__ constexpr int mono(int sigma, int c) {
    return ((sigma & 1) ^ (c == 0 ? 1 : 0)) | ((((sigma >> 1) & 1) ^ (c == 1 ? 1 : 0)) << 1) |
           ((((sigma >> 2) & 1) ^ (c == 2 ? 1 : 0)) << 2);
}

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

template <int NTH>
__device__ __forceinline__ double block_sum(double v, int tid) {
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

// ---------------------------------------------------------------------------
// Packed arithmetic.  A node value is held as V3 = {(u_x, u_y) as an f32x2
// pair, u_z}: every componentwise add or subtract is one packed instruction for
// x and y plus one scalar for z (sm_100+ FADD2 / FFMA2).  a - b is formed as
// fma(b, -1, a), which rounds exactly like the subtraction.
// ---------------------------------------------------------------------------
struct V3 {
    float2 xy;
    float z;
};
__device__ __forceinline__ V3 vadd(const V3& a, const V3& b) { return {__fadd2_rn(a.xy, b.xy), a.z + b.z}; }
__device__ __forceinline__ V3 vsub(const V3& a, const V3& b) {
    return {__ffma2_rn(b.xy, make_float2(-1.f, -1.f), a.xy), a.z - b.z};
}
__device__ __forceinline__ V3 vld(const float* p) { return {make_float2(p[0], p[1]), p[2]}; }
__device__ __forceinline__ float comp(const V3& v, int c) { return c == 0 ? v.xy.x : (c == 1 ? v.xy.y : v.z); }
__device__ __forceinline__ void set_comp(V3& v, int c, float x) {
    if (c == 0) v.xy.x = x;
    else if (c == 1) v.xy.y = x;
    else v.z = x;
}

// Difference sums of four corner values (x fastest), formed from node
// differences first: q[1] = x-difference, q[2] = y-difference, q[3] =
// xy-difference (signs of the corner coordinates).
__device__ __forceinline__ void face_diffs(const V3 c[4], V3 q[4]) {
    const V3 dx0 = vsub(c[1], c[0]), dx1 = vsub(c[3], c[2]);
    q[1] = vadd(dx0, dx1);
    q[2] = vadd(vsub(c[2], c[0]), vsub(c[3], c[1]));
    q[3] = vsub(dx1, dx0);
}

// State carried from one element layer to the next: the corners and the x/y
// difference sums of the shared face, and the top-face quantities of the layer.
struct Layer {
    V3 C[4];
    V3 Q[4];  // Q[0] unused
    V3 T[4];
    float E;
};

// 4-byte asynchronous global -> shared copy; when `valid` is false nothing is
// read and the destination is filled with zero.
__device__ __forceinline__ void cp_async4(unsigned dst, const float* gmem, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(gmem), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Ring slots of the shared-memory pipelines (lookahead 3 for planes and
// moduli, 2 for the epilogue operands, which are read one step late).  Slots are
// indexed by the step relative to the block's first layer.
constexpr int kRing = 4;

template <int BX, int BY, int MODE, bool DOT>
__global__ void __launch_bounds__(BX * BY, 2) k_fine(FineArgs a, GHat G, int zchunk) {
    constexpr int NT = BX * BY;
    constexpr int ROW = (BX + 1) * 3;           // floats per staged plane row
    constexpr int PLANE = (BY + 1) * ROW;       // floats per staged plane
    constexpr int NCP = (PLANE + NT - 1) / NT;  // plane copies per thread
    constexpr int OWN = (BX - 1) * (BY - 1);    // owned nodes per block
    constexpr bool EPI_B = MODE != FM_APPLY;
    constexpr bool EPI_D = MODE == FM_SMOOTH;
    __shared__ float sp[kRing][PLANE];                            // node planes
    __shared__ float sE[kRing][NT];                               // element moduli per layer
    __shared__ float sB[EPI_B ? kRing : 1][EPI_B ? OWN * 3 : 1];  // right-hand side at owned nodes
    __shared__ float sD[EPI_D ? kRing : 1][EPI_D ? OWN * 3 : 1];  // previous increment at owned nodes
    __shared__ float4 sx[2][BY][BX];                              // y-exchange: 3 row sums + modulus sum

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int nx = a.nx;
    const int NX = nx + 1, NY = a.ny + 1, NZ = a.nz + 1, NXY = NX * NY, NEXY = nx * a.ny;
    const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = blockIdx.z * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;                         // slot of plane / layer p is (p - kb) mod kRing
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;  // this column's cell; owned node (cx+1, cy+1)
    const int ox = cx + 1, oy = cy + 1;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const bool cell_in = cx >= 0 && cx < nx && cy >= 0 && cy < a.ny;
    const int onode_base = oy * NX + ox, e_base = cy * nx + cx;
    const int own3 = 3 * (ty * (BX - 1) + tx);  // owned-node slot inside the block (owners only)

    // per-thread plane copy slots: offset inside a global plane and validity
    int cp_goff[NCP];
    bool cp_ok[NCP];
#pragma unroll
    for (int q = 0; q < NCP; ++q) {
        const int idx = tid + q * NT;
        const int row = idx / ROW, c3 = idx % ROW;
        const int px = x0 - 1 + c3 / 3, py = y0 - 1 + row;
        cp_ok[q] = idx < PLANE && px >= 0 && px < NX && py >= 0 && py < NY;
        cp_goff[q] = cp_ok[q] ? 3 * (py * NX + px) + c3 % 3 : 0;
    }
    const unsigned sp_dst = smem_u32(&sp[0][tid]), sE_dst = smem_u32(&sE[0][tid]);
    const unsigned sB_dst = smem_u32(&sB[0][EPI_B ? own3 : 0]), sD_dst = smem_u32(&sD[0][EPI_D ? own3 : 0]);
    const float cd = EPI_D ? (float)a.coef[2 * a.step] : 0.f;
    const float ca = EPI_D ? (float)a.coef[2 * a.step + 1] : 0.f;
    const bool need_d = EPI_D && cd != 0.f;

    auto copy_plane = [&](int pz) {
        const bool zok = pz >= 0 && pz < NZ;
        const float* base = a.xin + 3 * (zok ? pz : 0) * NXY;
        const unsigned dst = sp_dst + 4u * (unsigned)(((pz - kb) & (kRing - 1)) * PLANE);
#pragma unroll
        for (int q = 0; q < NCP; ++q)
            if (tid + q * NT < PLANE) cp_async4(dst + 4u * q * NT, base + cp_goff[q], zok && cp_ok[q]);
    };
    // one commit group per step j: node plane j+4, modulus layer j+3, epilogue plane j+2
    auto issue = [&](int j) {
        if (j + 4 <= k1) copy_plane(j + 4);
        const int le = j + 3;
        if (le < k1) {
            const bool ok = cell_in && le >= 0 && le < a.nz;
            cp_async4(sE_dst + 4u * (unsigned)(((le - kb) & (kRing - 1)) * NT), a.E + (ok ? e_base + le * NEXY : 0),
                      ok);
        }
        const int pe = j + 2;
        if (EPI_B && owner && pe >= k0 && pe < k1) {
            const int slot = (pe - kb) & (kRing - 1);
            const float* src = a.b + 3 * (onode_base + pe * NXY);
            const unsigned db = sB_dst + 4u * (unsigned)(slot * OWN * 3);
            cp_async4(db, src, true);
            cp_async4(db + 4u, src + 1, true);
            cp_async4(db + 8u, src + 2, true);
            if (EPI_D && need_d) {
                const float* srd = a.dold + 3 * (onode_base + pe * NXY);
                const unsigned dd = sD_dst + 4u * (unsigned)(slot * OWN * 3);
                cp_async4(dd, srd, true);
                cp_async4(dd + 4u, srd + 1, true);
                cp_async4(dd + 8u, srd + 2, true);
            }
        }
        cp_commit();
    };
    // output masks of owned nodes, two planes ahead in registers
    auto load_mask = [&](int kp) -> uint8_t {
        return (owner && kp >= k0 && kp < k1) ? a.mask[onode_base + kp * NXY] : (uint8_t)7;
    };

    // ---- prologue: bottom plane k0-1 (own group), then the groups of steps k0-4 .. k0-2
    copy_plane(kb);
    cp_commit();
    issue(k0 - 4);
    issue(k0 - 3);
    issue(k0 - 2);
    uint8_t mk0 = 7, mk1 = load_mask(k0);  // masks of planes kl and kl+1 at step kl

    Layer s0, s1;
    asm volatile("cp.async.wait_group 3;\n" ::: "memory");
    __syncthreads();
    {
        const float* pl = sp[0];
        s0.C[0] = vld(pl + ty * ROW + 3 * tx);
        s0.C[1] = vld(pl + ty * ROW + 3 * tx + 3);
        s0.C[2] = vld(pl + (ty + 1) * ROW + 3 * tx);
        s0.C[3] = vld(pl + (ty + 1) * ROW + 3 * tx + 3);
        face_diffs(s0.C, s0.Q);
#pragma unroll
        for (int q = 0; q < 4; ++q) s0.T[q] = V3{make_float2(0.f, 0.f), 0.f};
        s0.E = 0.f;
    }
    bool pending = false;
    V3 R1{make_float2(0.f, 0.f), 0.f}, un_pend{make_float2(0.f, 0.f), 0.f};
    float eR1 = 0.f;
    uint8_t m_pend = 7;
    DSAcc dotv;

    // epilogue of the owned node of plane kp: its 4-cell sums R1 + the row above
    auto finish = [&](int kp) {
        const float4 up = sx[kp & 1][ty + 1][tx];
        const float y[3] = {R1.xy.x + up.x, R1.xy.y + up.y, R1.z + up.z};
        const int n = onode_base + kp * NXY;
        float* out = a.out + 3 * n;
        if (MODE == FM_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = fixed_bit(m_pend, c) ? 0.f : y[c];
                out[c] = v;
                if (DOT) dotv.add_prod(comp(un_pend, c), v);
            }
        } else {
            const int slot = (kp - kb) & (kRing - 1);
            const float* bb = &sB[EPI_B ? slot : 0][EPI_B ? own3 : 0];
            if (MODE == FM_RESID) {
#pragma unroll
                for (int c = 0; c < 3; ++c) out[c] = fixed_bit(m_pend, c) ? 0.f : bb[c] - y[c];
            } else {
                const float* dd = &sD[EPI_D ? slot : 0][EPI_D ? own3 : 0];
                const float inv = __frcp_rn(a.kd * (eR1 + up.w));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float xn = 0.f, dn = 0.f;
                    if (!fixed_bit(m_pend, c)) {
                        dn = ca * inv * (bb[c] - y[c]);
                        if (need_d) dn = fmaf(cd, dd[c], dn);
                        xn = comp(un_pend, c) + dn;
                        if (DOT) dotv.add_prod(bb[c], xn);
                    }
                    out[c] = xn;
                    if (a.dnew) a.dnew[3 * n + c] = dn;
                }
            }
        }
    };

    // one element layer kl: bottom face in `in`, top face into `out`
    auto layer = [&](const int kl, const Layer& in, Layer& out) {
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");  // group of step kl-3 has landed
        __syncthreads();
        if (pending && owner) finish(kl - 1);
        pending = false;
        issue(kl);  // overwrites the slots of plane kl and layer kl-1, last read in step kl-1
        const uint8_t mcur = mk0;
        mk0 = mk1;
        mk1 = load_mask(kl + 2);
        {
            const float* pl = sp[(kl + 1 - kb) & (kRing - 1)];
            out.C[0] = vld(pl + ty * ROW + 3 * tx);
            out.C[1] = vld(pl + ty * ROW + 3 * tx + 3);
            out.C[2] = vld(pl + (ty + 1) * ROW + 3 * tx);
            out.C[3] = vld(pl + (ty + 1) * ROW + 3 * tx + 3);
            face_diffs(out.C, out.Q);
        }
        out.E = sE[(kl - kb) & (kRing - 1)][tid];
        // modes: Z from per-corner z-differences, the others from the x/y
        // difference sums of the two faces
        V3 v[8];
        {
            const V3 z00 = vsub(out.C[0], in.C[0]), z10 = vsub(out.C[1], in.C[1]);
            const V3 z01 = vsub(out.C[2], in.C[2]), z11 = vsub(out.C[3], in.C[3]);
            v[4] = vadd(vadd(z00, z10), vadd(z01, z11));
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                v[q] = vadd(out.Q[q], in.Q[q]);
                v[q + 4] = vsub(out.Q[q], in.Q[q]);
            }
        }
        // w = E G v, class by class (the constant monomial carries no energy)
        V3 w[8];
        w[0] = V3{make_float2(0.f, 0.f), 0.f};
#pragma unroll
        for (int s = 0; s < 8; ++s) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int mi = mono(s, i);
                if (mi == 0) continue;
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int mj = mono(s, j);
                    if (mj == 0) continue;
                    acc = fmaf(G.g[s * 9 + i * 3 + j], comp(v[mj], j), acc);
                }
                set_comp(w[mi], i, acc);
            }
        }
        const float2 E2 = make_float2(out.E, out.E);
#pragma unroll
        for (int m = 1; m < 8; ++m) w[m] = V3{__fmul2_rn(E2, w[m].xy), out.E * w[m].z};
        // back to face quantities: top = w + w_z, bottom = w - w_z
        V3 Bf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out.T[q] = vadd(w[q], w[q + 4]);
            Bf[q] = vsub(w[q], w[q + 4]);
        }
        if (kl >= k0) {
            // plane kl is complete for this cell: S = top of layer kl-1 + bottom of
            // layer kl, expanded to the four corners and summed over the four cells
            // of each node (x by warp shuffle, y through shared memory)
            const V3 S0 = vadd(in.T[0], Bf[0]), S1 = vadd(in.T[1], Bf[1]);
            const V3 S2 = vadd(in.T[2], Bf[2]), S3 = vadd(in.T[3], Bf[3]);
            const V3 p = vsub(S0, S2), qd = vsub(S1, S3), r = vadd(S0, S2), sd = vadd(S1, S3);
            const V3 c00 = vsub(p, qd), c10 = vadd(p, qd), c01 = vsub(r, sd), c11 = vadd(r, sd);
            V3 n01, n00;
            n01.xy.x = __shfl_down_sync(0xffffffffu, c01.xy.x, 1, BX);
            n01.xy.y = __shfl_down_sync(0xffffffffu, c01.xy.y, 1, BX);
            n01.z = __shfl_down_sync(0xffffffffu, c01.z, 1, BX);
            n00.xy.x = __shfl_down_sync(0xffffffffu, c00.xy.x, 1, BX);
            n00.xy.y = __shfl_down_sync(0xffffffffu, c00.xy.y, 1, BX);
            n00.z = __shfl_down_sync(0xffffffffu, c00.z, 1, BX);
            R1 = vadd(c11, n01);
            const V3 r0 = vadd(c10, n00);
            const float es = in.E + out.E;
            const float er = es + __shfl_down_sync(0xffffffffu, es, 1, BX);
            sx[kl & 1][ty][tx] = make_float4(r0.xy.x, r0.xy.y, r0.z, er);
            pending = true;
            eR1 = er;
            un_pend = in.C[3];
            m_pend = mcur;
        }
    };

    // layers k0-1 .. k1-1, two per trip so that the layer state alternates
    // between s0 and s1 instead of being copied
    int kl = kb;
#pragma unroll 1
    for (; kl + 1 < k1; kl += 2) {
        layer(kl, s0, s1);
        layer(kl + 1, s1, s0);
    }
    if (kl < k1) layer(kl, s0, s1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    if (pending && owner) finish(k1 - 1);
    if (DOT) {
        const double s = block_sum<NT>(dotv.value(), tid);
        if (tid == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    }
}

// Copies x with the fixed DOFs of the fine level set to 0 (operands supplied by
// a caller may hold values there; the operator ignores them).
__global__ void k_mask_copy(const float* x, const uint8_t* mask, long long nn, float* out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * blockDim.x)
        out[q] = fixed_bit(mask[q / 3], (int)(q % 3)) ? 0.f : x[q];
}

// G = H K_e H^T / 64 restricted to the eight parity classes: g[s*9 + i*3 + j]
// couples component i of monomial mono(s, i) with component j of mono(s, j).
__global__ void k_hadamard_blocks(const double* Ke, double* g) {
    const int t = threadIdx.x;
    if (t >= 72) return;
    const int s = t / 9, i = (t / 3) % 3, j = t % 3;
    const int mi = mono(s, i), mj = mono(s, j);
    double acc = 0.0;
    for (int a = 0; a < 8; ++a) {
        const int sa = ((mi & 1) && !ldx(a) ? -1 : 1) * ((mi & 2) && !ldy(a) ? -1 : 1) * ((mi & 4) && !ldz(a) ? -1 : 1);
        for (int b = 0; b < 8; ++b) {
            const int sb = ((mj & 1) && !ldx(b) ? -1 : 1) * ((mj & 2) && !ldy(b) ? -1 : 1) * ((mj & 4) && !ldz(b) ? -1 : 1);
            acc += sa * sb * Ke[(3 * a + i) * 24 + 3 * b + j];
        }
    }
    g[t] = acc / 64.0;
}

struct FinePlan {
    int tile;   // 0: 32x8 threads (31x7 nodes), 1: 16x16 threads (15x15 nodes)
    int zc;     // node planes per block
    dim3 grid;
};

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

// Picks the tile shape and z-chunk length that minimise (waves x steps per
// block) for two resident blocks per SM: the partial tiles at the grid edges
// and the tail wave are the main losses on grids such as 101^3 nodes.
FinePlan plan_fine(int nx, int ny, int nz) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int slots = 2 * sm_count();
    FinePlan best{0, NZ, dim3(1, 1, 1)};
    long long best_cost = -1;
    const int shapes[2][2] = {{32, 8}, {16, 16}};
    for (int t = 0; t < 2; ++t) {
        const int bx = shapes[t][0], by = shapes[t][1];
        const int gx = (NX + bx - 2) / (bx - 1), gy = (NY + by - 2) / (by - 1);
        for (int nch = 1; nch <= NZ; ++nch) {
            const int zc = (NZ + nch - 1) / nch;
            if (zc < 4 && nch > 1) break;
            const int gz = (NZ + zc - 1) / zc;
            const long long blocks = (long long)gx * gy * gz;
            const long long waves = (blocks + slots - 1) / slots;
            const long long cost = waves * (zc + 1) * 64 + (blocks % slots == 0 ? 0 : 1);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best = FinePlan{t, zc, dim3(gx, gy, gz)};
            }
        }
    }
    return best;
}

template <int MODE, bool DOT>
void launch_shape(const FinePlan& pl, const FineArgs& a, const GHat& G, cudaStream_t s) {
    if (pl.tile == 0) k_fine<32, 8, MODE, DOT><<<pl.grid, dim3(32, 8), 0, s>>>(a, G, pl.zc);
    else k_fine<16, 16, MODE, DOT><<<pl.grid, dim3(16, 16), 0, s>>>(a, G, pl.zc);
}

}  // namespace

int fine_grid_blocks(int nx, int ny, int nz) {
    const FinePlan pl = plan_fine(nx, ny, nz);
    return (int)(pl.grid.x * pl.grid.y * pl.grid.z);
}

void launch_fine(int mode, int dot, int mask_in, const FineArgs& a_in, const GHat& G, cudaStream_t s) {
    const FinePlan pl = plan_fine(a_in.nx, a_in.ny, a_in.nz);
    FineArgs a = a_in;
    if (mask_in && a.scratch) {
        const long long nn = (long long)(a.nx + 1) * (a.ny + 1) * (a.nz + 1);
        note_launch();
        k_mask_copy<<<(int)std::min<long long>((3 * nn + 255) / 256, 148 * 8), 256, 0, s>>>(a.xin, a.mask, nn,
                                                                                             a.scratch);
        a.xin = a.scratch;
    }
    note_launch();
    if (mode == FM_APPLY) {
        if (dot) launch_shape<FM_APPLY, true>(pl, a, G, s);
        else launch_shape<FM_APPLY, false>(pl, a, G, s);
    } else if (mode == FM_SMOOTH) {
        if (dot) launch_shape<FM_SMOOTH, true>(pl, a, G, s);
        else launch_shape<FM_SMOOTH, false>(pl, a, G, s);
    } else {
        launch_shape<FM_RESID, false>(pl, a, G, s);
    }
}

void launch_hadamard_blocks(const double* Ke, double* g72, cudaStream_t s) {
    note_launch();
    k_hadamard_blocks<<<1, 96, 0, s>>>(Ke, g72);
}

}  // namespace gmg
