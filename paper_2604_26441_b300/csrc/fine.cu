// Matrix-free fine-level operator (Eq. mf_matvec) fused with its consumers, for sm_103a.
//
// Formulation.  On the unit cube the 24x24 element stiffness K_e commutes with
// the reflections x -> 1-x, y -> 1-y, z -> 1-z.  In the basis of the eight
// monomials {1, X, Y, Z, XY, YZ, XZ, XYZ} of the corner signs (an 8-point
// Walsh-Hadamard transform H of the node values, per displacement component)
// it is block diagonal: the parity of (monomial, component) under the three
// reflections splits the 24 modes into 8 classes of 3, and
//     K_e = H^T G H,  G = H K_e H^T / 64,
// with G made of eight 3x3 blocks (72 numbers; the constant monomial is a
// rigid translation and drops out).  The symmetry of the cube under axis
// permutations leaves eight distinct values in those blocks (GSym in
// internal.cuh), so with E_e folded into the eight, one element application
// costs 21 mode sums, 8 coefficient products and 33 operations for G instead of
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
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

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
__device__ __forceinline__ V3 vadd(const V3& a, const V3& b) { return {__fadd2_rn(a.xy, b.xy), __fadd_rn(a.z, b.z)}; }
__device__ __forceinline__ V3 vsub(const V3& a, const V3& b) {
    return {__ffma2_rn(b.xy, make_float2(-1.f, -1.f), a.xy), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ V3 vld(const float* p) { return {make_float2(p[0], p[1]), p[2]}; }
__device__ __forceinline__ float comp(const V3& v, int c) { return c == 0 ? v.xy.x : (c == 1 ? v.xy.y : v.z); }

// w[1..7] = E_e G v[1..7] for one element (GSym form of G, E_e in k).
__device__ __forceinline__ void contract_v3(const GElem<float>& k, const V3 (&v)[8], V3 (&w)[8]) {
    float u[8][3], o[8][3];
#pragma unroll
    for (int m = 1; m < 8; ++m) {
        u[m][0] = v[m].xy.x;
        u[m][1] = v[m].xy.y;
        u[m][2] = v[m].z;
    }
    gsym_contract(k, u, o);
#pragma unroll
    for (int m = 1; m < 8; ++m) w[m] = V3{make_float2(o[m][0], o[m][1]), o[m][2]};
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
__global__ void __launch_bounds__(BX * BY, 2) k_fine(FineArgs a, GSym G, int zchunk) {
    pdl_entry();
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
    const int NX = nx + 1, NY = a.ny + 1, NZ = a.nz + 1, NEXY = nx * a.ny;
    const int PX = a.pitch ? a.pitch : NX, NXY = PX * NY;  // vectors and mask: PX nodes per row
    const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = blockIdx.z * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;                         // slot of plane / layer p is (p - kb) mod kRing
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;  // this column's cell; owned node (cx+1, cy+1)
    const int ox = cx + 1, oy = cy + 1;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const bool cell_in = cx >= 0 && cx < nx && cy >= 0 && cy < a.ny;
    const int onode_base = oy * PX + ox, e_base = cy * nx + cx;
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
        cp_goff[q] = cp_ok[q] ? 3 * (py * PX + px) + c3 % 3 : 0;
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
        return (owner && kp >= k0 && kp < k1) ? a.mask[GMG_B(onode_base + kp * NXY, (long long)NXY * NZ, 111)] : (uint8_t)7;
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
        const float y[3] = {__fadd_rn(R1.xy.x, up.x), __fadd_rn(R1.xy.y, up.y), __fadd_rn(R1.z, up.z)};
        const long long n = GMG_B(onode_base + kp * NXY, (long long)NXY * NZ, 112);
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
                for (int c = 0; c < 3; ++c) out[c] = fixed_bit(m_pend, c) ? 0.f : __fsub_rn(bb[c], y[c]);
            } else {
                const float* dd = &sD[EPI_D ? slot : 0][EPI_D ? own3 : 0];
                const float inv = jacobi_rcp(__fmul_rn(a.kd, __fadd_rn(eR1, up.w)));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float xn = 0.f, dn = 0.f;
                    if (!fixed_bit(m_pend, c)) {
                        dn = __fmul_rn(__fmul_rn(ca, inv), __fsub_rn(bb[c], y[c]));
                        if (need_d) dn = fmaf(cd, dd[c], dn);
                        xn = __fadd_rn(comp(un_pend, c), dn);
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
        // w = E G v (the constant monomial carries no energy)
        V3 w[8];
        w[0] = V3{make_float2(0.f, 0.f), 0.f};
        contract_v3(gsym_scale(G, out.E), v, w);
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
            const float es = __fadd_rn(in.E, out.E);
            const float er = __fadd_rn(es, __shfl_down_sync(0xffffffffu, es, 1, BX));
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

// ---------------------------------------------------------------------------
// Tensor-core smoother (the precision line of Sec. "Mixed precision"): the
// same z-marching smoother step, with the element contraction on the 5th-gen
// tensor cores.  Per element layer every thread forms its element's 21 Hadamard
// modes in FP32 (as above; differences, so the low-precision rounding acts on
// the variation of u), splits them into BF16 hi (+ lo) parts and writes one row
// of a 128 x 32 BF16 A tile in shared memory.  One thread issues
// tcgen05.mma (kind::f16, FP32 accumulation in TMEM) against the fixed 32 x 32
// operand B that maps the 21 modes to the 24 corner forces of the element (G
// composed with the face split and the corner expansion, built on the host in
// FP64 and split into BF16 hi + lo).  PASSES = 1: A_hi B_hi (plain BF16);
// PASSES = 3: + A_lo B_hi + A_hi B_lo (split BF16, ~16 significant bits).  The
// result of layer k is read back from TMEM one step later (tcgen05.ld), scaled
// by E_e in FP32 and summed into the nodes as above; node plane p is finished
// three steps after its layer, so the epilogue operands are loaded one plane
// earlier than in k_fine.
// ---------------------------------------------------------------------------
constexpr int kTcTileBytes = 128 * 32 * 2;  // one 128 x 32 BF16 operand tile
constexpr unsigned kTcSpin = 1u << 22;

__device__ __forceinline__ uint64_t tc_sdesc(unsigned addr) {
    // K-major, no swizzle: core matrices of 8 rows x 16 bytes; K-adjacent cores
    // 128 bytes apart (leading offset), row-group-adjacent cores 512 bytes apart
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// byte offset of (row r, k-chunk j of 8 BF16 values) in a tile
__device__ __forceinline__ int tc_chunk(int r, int j) { return ((r >> 3) * 4 + j) * 128 + (r & 7) * 16; }

__device__ __forceinline__ unsigned bf2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&b);
}
__device__ __forceinline__ float2 unbf2(unsigned u) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}

template <int BX, int BY, int PASSES, bool DOT>
__global__ void __launch_bounds__(BX * BY, 2) k_fine_tc(FineArgs a, int zchunk) {
    static_assert(BX * BY == 256, "two 128-element MMA tiles per block");
    constexpr int NT = BX * BY;
    constexpr int ROW = (BX + 1) * 3;
    constexpr int PLANE = (BY + 1) * ROW;
    constexpr int NCP = (PLANE + NT - 1) / NT;
    constexpr int OWN = (BX - 1) * (BY - 1);
    constexpr int APARTS = PASSES > 1 ? 2 : 1;
    __shared__ float sp[kRing][PLANE];
    __shared__ float sE[kRing][NT];
    __shared__ float sB[kRing][OWN * 3];
    __shared__ float sD[kRing][OWN * 3];
    __shared__ float4 sx[2][BY][BX];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ unsigned tslot;
    extern __shared__ __align__(1024) unsigned char dyn[];  // A tiles [APARTS][2], then B [2]
    unsigned char* const sA = dyn;
    unsigned char* const sBop = dyn + APARTS * 2 * kTcTileBytes;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty, warp = tid >> 5;
    const int nx = a.nx;
    const int NX = nx + 1, NY = a.ny + 1, NZ = a.nz + 1, NEXY = nx * a.ny;
    const int PX = a.pitch ? a.pitch : NX, NXY = PX * NY;  // vectors and mask: PX nodes per row
    const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = blockIdx.z * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty, ox = cx + 1, oy = cy + 1;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const bool cell_in = cx >= 0 && cx < nx && cy >= 0 && cy < a.ny;
    const int onode_base = oy * PX + ox, e_base = cy * nx + cx;
    const int own3 = 3 * (ty * (BX - 1) + tx);
    const int trow = tid & 127, ttile = tid >> 7;  // this element's row and tile in the MMA

    if ((smem_u32(dyn) & 1023) != 0) {  // operand tiles must be 16-byte (here 1 KB) aligned
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    // ---- operand B into shared memory, A pad columns (k 24..31) to zero, TMEM, barriers
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tcB);
        uint4* dst = reinterpret_cast<uint4*>(sBop);
        for (int q = tid; q < 2 * 2048 / 16; q += NT) dst[q] = src[q];
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int pa = 0; pa < APARTS; ++pa)
            *reinterpret_cast<uint4*>(sA + (pa * 2 + ttile) * kTcTileBytes + tc_chunk(trow, 3)) = z;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }

    int cp_goff[NCP];
    bool cp_ok[NCP];
#pragma unroll
    for (int q = 0; q < NCP; ++q) {
        const int idx = tid + q * NT;
        const int row = idx / ROW, c3 = idx % ROW;
        const int px = x0 - 1 + c3 / 3, py = y0 - 1 + row;
        cp_ok[q] = idx < PLANE && px >= 0 && px < NX && py >= 0 && py < NY;
        cp_goff[q] = cp_ok[q] ? 3 * (py * PX + px) + c3 % 3 : 0;
    }
    const unsigned sp_dst = smem_u32(&sp[0][tid]), sE_dst = smem_u32(&sE[0][tid]);
    const unsigned sB_dst = smem_u32(&sB[0][own3]), sD_dst = smem_u32(&sD[0][own3]);
    const float cd = (float)a.coef[2 * a.step], ca = (float)a.coef[2 * a.step + 1];
    const bool need_d = cd != 0.f;

    auto copy_plane = [&](int pz) {
        const bool zok = pz >= 0 && pz < NZ;
        const float* base = a.xin + 3 * (zok ? pz : 0) * NXY;
        const unsigned dst = sp_dst + 4u * (unsigned)(((pz - kb) & (kRing - 1)) * PLANE);
#pragma unroll
        for (int q = 0; q < NCP; ++q)
            if (tid + q * NT < PLANE) cp_async4(dst + 4u * q * NT, base + cp_goff[q], zok && cp_ok[q]);
    };
    // group j: node plane j+4, modulus layer j+3, epilogue operands of plane j+1
    auto issue = [&](int j) {
        if (j + 4 <= k1) copy_plane(j + 4);
        const int le = j + 3;
        if (le < k1) {
            const bool ok = cell_in && le >= 0 && le < a.nz;
            cp_async4(sE_dst + 4u * (unsigned)(((le - kb) & (kRing - 1)) * NT), a.E + (ok ? e_base + le * NEXY : 0),
                      ok);
        }
        const int pe = j + 1;
        if (owner && pe >= k0 && pe < k1) {
            const int slot = (pe - kb) & (kRing - 1);
            const float* src = a.b + 3 * (onode_base + pe * NXY);
            const unsigned db = sB_dst + 4u * (unsigned)(slot * OWN * 3);
            cp_async4(db, src, true);
            cp_async4(db + 4u, src + 1, true);
            cp_async4(db + 8u, src + 2, true);
            if (need_d) {
                const float* srd = a.dold + 3 * (onode_base + pe * NXY);
                const unsigned dd = sD_dst + 4u * (unsigned)(slot * OWN * 3);
                cp_async4(dd, srd, true);
                cp_async4(dd + 4u, srd + 1, true);
                cp_async4(dd + 8u, srd + 2, true);
            }
        }
        cp_commit();
    };
    auto load_mask = [&](int kp) -> uint8_t {
        return (owner && kp >= k0 && kp < k1) ? a.mask[onode_base + kp * NXY] : (uint8_t)7;
    };

    // ---- prologue (as k_fine; one more epilogue group ahead)
    copy_plane(kb);
    cp_commit();
    issue(k0 - 4);
    issue(k0 - 3);
    issue(k0 - 2);
    asm volatile("cp.async.wait_group 3;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tslot;
    const unsigned a_base = smem_u32(sA), b_base = smem_u32(sBop);
    // TMEM address of this thread's row in buffer `buf`, tile `ttile`: lanes 32*(warp%4).., columns (buf*2+tile)*32
    const unsigned my_d = tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(ttile * 32);

    Layer L0, L1;
    {
        const float* pl = sp[0];
        L0.C[0] = vld(pl + ty * ROW + 3 * tx);
        L0.C[1] = vld(pl + ty * ROW + 3 * tx + 3);
        L0.C[2] = vld(pl + (ty + 1) * ROW + 3 * tx);
        L0.C[3] = vld(pl + (ty + 1) * ROW + 3 * tx + 3);
        face_diffs(L0.C, L0.Q);
    }
    // pipelines: E of the last three layers, x of the owned node at the last three
    // planes, masks of the next planes
    float e_h0 = 0.f, e_h1 = 0.f, e_h2 = 0.f, e_prevc = 0.f;
    V3 u_h0{make_float2(0.f, 0.f), 0.f}, u_h1 = u_h0, u_h2 = u_h0, un_pend = u_h0;
    uint8_t m_h0 = 7, m_h1 = 7, m_pend = 7;
    V3 topPrev[4], R1 = u_h0;
#pragma unroll
    for (int q = 0; q < 4; ++q) topPrev[q] = u_h0;
    float eR1 = 0.f;
    bool pending = false;
    int pend_k = 0;
    bool failed = false;
    DSAcc dotv;

    auto wait_mma = [&](int p) -> bool {
        const int g = p - kb;
        for (unsigned it = 0; it < kTcSpin; ++it)
            if (mbar_try_wait(&mbar[g & 1], (g >> 1) & 1)) return true;
        return false;
    };
    auto finish = [&](int kp) {
        const float4 up = sx[kp & 1][ty + 1][tx];
        const float y[3] = {__fadd_rn(R1.xy.x, up.x), __fadd_rn(R1.xy.y, up.y), __fadd_rn(R1.z, up.z)};
        const int n = onode_base + kp * NXY;
        float* out = a.out + 3 * n;
        const int slot = (kp - kb) & (kRing - 1);
        const float* bb = &sB[slot][own3];
        const float* dd = &sD[slot][own3];
        const float inv = jacobi_rcp(__fmul_rn(a.kd, __fadd_rn(eR1, up.w)));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float xn = 0.f, dn = 0.f;
            if (!fixed_bit(m_pend, c)) {
                dn = __fmul_rn(__fmul_rn(ca, inv), __fsub_rn(bb[c], y[c]));
                if (need_d) dn = fmaf(cd, dd[c], dn);
                xn = __fadd_rn(comp(un_pend, c), dn);
                if (DOT) dotv.add_prod(bb[c], xn);
            }
            out[c] = xn;
            if (a.dnew) a.dnew[3 * n + c] = dn;
        }
    };

    // step s: MMA of layer s-1, epilogue of plane s-3, modes of layer s, node
    // sums of plane s-2 (from the MMA of layer s-2)
    auto step = [&](const int s, const Layer& in, Layer& out) {
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int p1 = s - 1;
        if (tid == 0 && p1 >= kb && p1 < k1) {
            constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
            const unsigned dbuf = tmem + (unsigned)(((p1 - kb) & 1) * 64);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
#pragma unroll
                for (int pass = 0; pass < PASSES; ++pass) {
                    const int apart = pass == 1 ? 1 : 0, bpart = pass == 2 ? 1 : 0;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t da = tc_sdesc(a_base + (apart * 2 + t) * kTcTileBytes + ks * 256);
                        const uint64_t db = tc_sdesc(b_base + bpart * 2048 + ks * 256);
                        const unsigned acc = (pass > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dbuf + t * 32),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[(p1 - kb) & 1]))
                         : "memory");
        }
        if (pending && owner) finish(pend_k);
        pending = false;
        issue(s);
        // pipelines
        m_h1 = m_h0;
        m_h0 = load_mask(s - 1);
        e_h2 = e_h1;
        e_h1 = e_h0;
        u_h2 = u_h1;
        u_h1 = u_h0;
        u_h0 = in.C[3];
        if (s < k1) {
            // modes of layer s (bottom face in `in`, top plane s+1 from the ring)
            const float* pl = sp[(s + 1 - kb) & (kRing - 1)];
            out.C[0] = vld(pl + ty * ROW + 3 * tx);
            out.C[1] = vld(pl + ty * ROW + 3 * tx + 3);
            out.C[2] = vld(pl + (ty + 1) * ROW + 3 * tx);
            out.C[3] = vld(pl + (ty + 1) * ROW + 3 * tx + 3);
            face_diffs(out.C, out.Q);
            e_h0 = cell_in ? sE[(s - kb) & (kRing - 1)][tid] : 0.f;
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
            // the A tile is free once the MMA of layer s-1 has completed
            if (p1 >= kb && !wait_mma(p1)) failed = true;
            float m21[22];
#pragma unroll
            for (int m = 1; m < 8; ++m) {
                m21[3 * (m - 1)] = v[m].xy.x;
                m21[3 * (m - 1) + 1] = v[m].xy.y;
                m21[3 * (m - 1) + 2] = v[m].z;
            }
            m21[21] = 0.f;
            unsigned hi[11], lo[11];
#pragma unroll
            for (int q = 0; q < 11; ++q) {
                hi[q] = bf2(m21[2 * q], m21[2 * q + 1]);
                if (PASSES > 1) {
                    const float2 h = unbf2(hi[q]);
                    lo[q] = bf2(m21[2 * q] - h.x, m21[2 * q + 1] - h.y);
                }
            }
            unsigned char* at = sA + ttile * kTcTileBytes;
            *reinterpret_cast<uint4*>(at + tc_chunk(trow, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(at + tc_chunk(trow, 1)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
            *reinterpret_cast<uint4*>(at + tc_chunk(trow, 2)) = make_uint4(hi[8], hi[9], hi[10], 0u);
            if (PASSES > 1) {
                unsigned char* al = sA + (2 + ttile) * kTcTileBytes;
                *reinterpret_cast<uint4*>(al + tc_chunk(trow, 0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<uint4*>(al + tc_chunk(trow, 1)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                *reinterpret_cast<uint4*>(al + tc_chunk(trow, 2)) = make_uint4(lo[8], lo[9], lo[10], 0u);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        // node sums of plane p = s-2 from the corner forces of layer p
        const int p = s - 2;
        if (p >= kb && p < k1) {
            if (!wait_mma(p)) failed = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned d[24];
            const unsigned taddr = my_d + (unsigned)(((p - kb) & 1) * 64);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                  "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
                : "r"(taddr));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]),
                           "=r"(d[23])
                         : "r"(taddr + 16u));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const float E = e_h2;
            const float2 E2 = make_float2(E, E);
            V3 bot[4], top[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                bot[q] = V3{__fmul2_rn(E2, make_float2(__uint_as_float(d[3 * q]), __uint_as_float(d[3 * q + 1]))),
                            E * __uint_as_float(d[3 * q + 2])};
                top[q] = V3{__fmul2_rn(E2, make_float2(__uint_as_float(d[12 + 3 * q]), __uint_as_float(d[13 + 3 * q]))),
                            E * __uint_as_float(d[14 + 3 * q])};
            }
            if (p >= k0) {
                const V3 c00 = vadd(topPrev[0], bot[0]), c10 = vadd(topPrev[1], bot[1]);
                const V3 c01 = vadd(topPrev[2], bot[2]), c11 = vadd(topPrev[3], bot[3]);
                V3 n01, n00;
                n01.xy.x = __shfl_down_sync(0xffffffffu, c01.xy.x, 1, BX);
                n01.xy.y = __shfl_down_sync(0xffffffffu, c01.xy.y, 1, BX);
                n01.z = __shfl_down_sync(0xffffffffu, c01.z, 1, BX);
                n00.xy.x = __shfl_down_sync(0xffffffffu, c00.xy.x, 1, BX);
                n00.xy.y = __shfl_down_sync(0xffffffffu, c00.xy.y, 1, BX);
                n00.z = __shfl_down_sync(0xffffffffu, c00.z, 1, BX);
                R1 = vadd(c11, n01);
                const V3 r0 = vadd(c10, n00);
                const float es = __fadd_rn(e_prevc, E);
                const float er = __fadd_rn(es, __shfl_down_sync(0xffffffffu, es, 1, BX));
                sx[p & 1][ty][tx] = make_float4(r0.xy.x, r0.xy.y, r0.z, er);
                pending = true;
                pend_k = p;
                eR1 = er;
                un_pend = u_h2;
                m_pend = m_h1;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) topPrev[q] = top[q];
            e_prevc = E;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    int s = kb;
#pragma unroll 1
    for (; s + 1 <= k1 + 2; s += 2) {
        step(s, L0, L1);
        step(s + 1, L1, L0);
        if (__syncthreads_or(failed)) break;
    }
    if (!failed && s <= k1 + 2) step(s, L0, L1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const bool bad = __syncthreads_or(failed);
    if (!bad && pending && owner) finish(pend_k);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    if (bad) {
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    if (DOT) {
        const double sum = block_sum<NT>(dotv.value(), tid);
        if (tid == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = sum;
    }
}

// ---------------------------------------------------------------------------
// TMA-fed fine operator (the default for the solver's own level-0 vectors).
// Same element arithmetic and z-march as k_fine, but every operand tile of a
// step arrives by tiled TMA (cp.async.bulk.tensor) issued by one thread on one
// mbarrier per ring slot, instead of per-thread 4-byte copies with their
// address and predicate work.  This needs the level-0 vectors in the padded
// layout [NZ][NY][px][3] with px (nodes per row) a multiple of 4, so every node
// row starts on a 16-byte boundary, and the moduli in [nz][ny][ex] with ex a
// multiple of 4.  A box's innermost coordinate is rounded down to a multiple of
// 4 floats; the block reads its tile at a constant offset (0..3 floats) inside
// the box.  Boxes reaching outside the grid read zeros (TMA fill), so there are
// no edge predicates on the staged data.
//
// Stage s (ring slot (s - kb) mod 4) holds: node plane s+1 (the top face of
// layer s), moduli layer s, and the epilogue operands (b, previous increment)
// of node plane s-1, which is finished at step s.  Stage s is issued at step
// s-3, right after the block barrier that ends the reads of the slot's previous
// stage.  The loop takes four steps per trip, so ring slots are compile-time
// offsets and the mbarrier phase is one bit per trip.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int round4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int round128(int v) { return (v + 127) / 128 * 128; }
__device__ __forceinline__ int floor4(int v) { return v & ~3; }  // two's complement: rounds toward -inf

template <int BX, int BY>
struct TmaTile {
    static constexpr int XW = round4(3 * (BX + 1) + 3);  // floats per staged node row (+ up to 3 of offset)
    static constexpr int XR = BY + 1;                    // node rows
    static constexpr int EW = round4(BX + 3);            // moduli per staged row
    static constexpr int ER = BY;
    static constexpr int OW = round4(3 * (BX - 1) + 3);  // floats per row of owned nodes
    static constexpr int OR = BY - 1;
    static constexpr int XB = XW * XR * 4, EB = EW * ER * 4, OB = OW * OR * 4;
    static constexpr int XOFF = 0;
    static constexpr int EOFF = round128(XB);
    static constexpr int BOFF = EOFF + round128(EB);
    static constexpr int DOFF = BOFF + round128(OB);
    static constexpr int STAGE = DOFF + round128(OB);
    static constexpr int SXOFF = 4 * STAGE;              // y-exchange [2][BY + 1][BX] float4 (row BY unused)
    static constexpr int BAROFF = SXOFF + 2 * (BY + 1) * BX * 16;
    static constexpr int SMEM = BAROFF + 4 * 8;
};

constexpr unsigned kTmaSpin = 1u << 22;

template <int BX, int BY, int MODE, bool DOT>
__global__ void __launch_bounds__(BX * BY, 2)
k_fine_tma(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tme,
           const __grid_constant__ CUtensorMap tmb, const __grid_constant__ CUtensorMap tmd, FineArgs a, GSym G,
           int zchunk) {
    using T = TmaTile<BX, BY>;
    constexpr int NT = BX * BY;
    constexpr bool EPI_B = MODE != FM_APPLY;
    constexpr bool EPI_D = MODE == FM_SMOOTH;
    extern __shared__ __align__(128) unsigned char smem[];
    float4(*sx)[BY + 1][BX] = reinterpret_cast<float4(*)[BY + 1][BX]>(smem + T::SXOFF);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + T::BAROFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int px = a.pitch, NXYp = px * NY;
    const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = blockIdx.z * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;
    // box origins (innermost coordinate rounded down to 4 floats) and offsets
    const int xs = floor4(3 * (x0 - 1)), es = floor4(x0 - 1), bs = floor4(3 * x0);
    const int rx = ty * T::XW + 3 * tx + (3 * (x0 - 1) - xs);  // this column's low corner in a node plane
    const int re = ty * T::EW + tx + (x0 - 1 - es);            // this column's modulus in a layer
    const int rb = ty * T::OW + 3 * tx + (3 * x0 - bs);        // this owner's node in an epilogue plane
    const int ox = x0 + tx, oy = y0 + ty;
    const bool owner = tx < BX - 1 && ty < BY - 1 && ox < NX && oy < NY;
    const int onode = oy * px + ox;
    const float cd = EPI_D ? (float)a.coef[2 * a.step] : 0.f;
    const float ca = EPI_D ? (float)a.coef[2 * a.step + 1] : 0.f;
    const bool need_d = EPI_D && cd != 0.f;
    const unsigned epi_bytes = EPI_B ? (unsigned)T::OB * (need_d ? 2u : 1u) : 0u;

    if ((smem_u32(smem) & 127) != 0) {  // TMA destinations are laid out on 128-byte boundaries
        if (tid == 0) atomicExch(a.err, 1);
        return;
    }
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) mbar_init(&full[q], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // Everything above ran before the previous kernel finished (programmatic
    // dependent launch); the operands may only be read from here on.
    pdl_entry();

    // stage s into its ring slot (thread 0 only); stages past the chunk's last
    // read are skipped, and so are their waits.  issued[q] counts the phases
    // started on slot q (thread 0's copy only), for the failure path.
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
            tma_load_3d(st + T::XOFF, &tmx, xs, y0 - 1, s + 1, &full[q]);
            tma_load_3d(st + T::EOFF, &tme, es, y0 - 1, s, &full[q]);
        }
        if (ep) {
            tma_load_3d(st + T::BOFF, &tmb, bs, y0, s - 1, &full[q]);
            if (need_d) tma_load_3d(st + T::DOFF, &tmd, bs, y0, s - 1, &full[q]);
        }
    };
    auto wait_full = [&](int q, unsigned parity) -> bool {
        for (unsigned it = 0; it < kTmaSpin; ++it)
            if (mbar_try_wait(&full[q], parity)) return true;
        return false;
    };
    // masks held as int (no byte packing); non-owners see every DOF fixed
    auto load_mask = [&](int kp) -> int {
        return (owner && kp >= k0 && kp < k1) ? (int)a.mask[GMG_B(onode + kp * NXYp, (long long)NXYp * NZ, 101)] : 7;
    };

    // ---- prologue: bottom plane kb into slot 3's plane region (its first phase),
    // stages kb .. kb+2 into slots 0..2
    if (tid == 0) {
        issued[3] = 1;
        mbar_expect_tx(&full[3], (unsigned)T::XB);
        tma_load_3d(smem + 3 * T::STAGE + T::XOFF, &tmx, xs, y0 - 1, kb, &full[3]);
        issue(kb);
        if (kb + 1 <= k1) issue(kb + 1);
        if (kb + 2 <= k1) issue(kb + 2);
    }
    bool failed = !wait_full(3, 0);
    Layer s0, s1;
    {
        const float* pl = reinterpret_cast<const float*>(smem + 3 * T::STAGE + T::XOFF) + rx;
        s0.C[0] = vld(pl);
        s0.C[1] = vld(pl + 3);
        s0.C[2] = vld(pl + T::XW);
        s0.C[3] = vld(pl + T::XW + 3);
        face_diffs(s0.C, s0.Q);
#pragma unroll
        for (int q = 0; q < 4; ++q) s0.T[q] = V3{make_float2(0.f, 0.f), 0.f};
        s0.E = 0.f;
    }
    // masks four planes ahead, one register per ring slot (the slot of step s
    // holds plane s's mask), so a load's result is not touched before its use
    int mq[4] = {7, load_mask(k0), load_mask(k0 + 1), load_mask(k0 + 2)};
    bool pending = false;
    V3 R1{make_float2(0.f, 0.f), 0.f}, un_pend{make_float2(0.f, 0.f), 0.f};
    float eR1 = 0.f;
    int m_pend = 7;
    DSAcc dotv;

    // Epilogue of the owned node of plane kp from the stage in slot q.  Every
    // thread runs it without branches (non-owners hold an all-fixed mask, so
    // their values are zeros or discarded); only the stores are predicated.
    auto finish = [&](int kp, int q) {
        const float4 up = sx[kp & 1][ty + 1][tx];
        const float y[3] = {__fadd_rn(R1.xy.x, up.x), __fadd_rn(R1.xy.y, up.y), __fadd_rn(R1.z, up.z)};
        const long long on = owner ? GMG_B(onode + kp * NXYp, (long long)NXYp * NZ, 102) : 0;
        float* out = a.out + 3 * on;
        if (MODE == FM_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fr = !fixed_bit(m_pend, c);
                const float v = fr ? y[c] : 0.f;
                if (owner) out[c] = v;
                if (DOT) dotv.add_prod(fr ? comp(un_pend, c) : 0.f, v);
            }
        } else {
            const float* bb = reinterpret_cast<const float*>(smem + q * T::STAGE + T::BOFF) + rb;
            if (MODE == FM_RESID) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = fixed_bit(m_pend, c) ? 0.f : __fsub_rn(bb[c], y[c]);
                    if (owner) out[c] = v;
                }
            } else {
                const float* dd = reinterpret_cast<const float*>(smem + q * T::STAGE + T::DOFF) + rb;
                const float inv = jacobi_rcp(__fmul_rn(a.kd, __fadd_rn(eR1, up.w)));
                float* dn_out = a.dnew + 3 * on;
                const bool wd = owner && a.dnew != nullptr;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const bool fr = !fixed_bit(m_pend, c);
                    float dn = __fmul_rn(__fmul_rn(ca, inv), __fsub_rn(bb[c], y[c]));
                    if (need_d) dn = fmaf(cd, dd[c], dn);
                    dn = fr ? dn : 0.f;
                    const float xn = fr ? __fadd_rn(comp(un_pend, c), dn) : 0.f;
                    if (DOT) dotv.add_prod(fr ? bb[c] : 0.f, xn);
                    if (owner) out[c] = xn;
                    if (wd) dn_out[c] = dn;
                }
            }
        }
    };

    // one step s = one element layer (bottom face in `in`, top face into `out`)
    // with the stage in slot Q; `par` is the trip's phase bit
    auto step = [&](auto Qc, const int s, const unsigned par, const Layer& in, Layer& out) -> bool {
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
            out.C[0] = vld(pl);
            out.C[1] = vld(pl + 3);
            out.C[2] = vld(pl + T::XW);
            out.C[3] = vld(pl + T::XW + 3);
            face_diffs(out.C, out.Q);
        }
        out.E = reinterpret_cast<const float*>(smem + Q * T::STAGE + T::EOFF)[re];
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
        V3 w[8];
        w[0] = V3{make_float2(0.f, 0.f), 0.f};
        contract_v3(gsym_scale(G, out.E), v, w);
        V3 Bf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out.T[q] = vadd(w[q], w[q + 4]);
            Bf[q] = vsub(w[q], w[q + 4]);
        }
        if (s >= k0) {
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

    // layers kb .. k1-1, four per trip (slots 0..3 in order), the layer state
    // alternating between s0 and s1
    unsigned par = 0;
    bool ok = !failed;
    for (int s = kb; ok && s < k1; s += 4, par ^= 1u) {
        ok = step(std::integral_constant<int, 0>{}, s, par, s0, s1);
        if (ok && s + 1 < k1) ok = step(std::integral_constant<int, 1>{}, s + 1, par, s1, s0);
        if (ok && s + 2 < k1) ok = step(std::integral_constant<int, 2>{}, s + 2, par, s0, s1);
        if (ok && s + 3 < k1) ok = step(std::integral_constant<int, 3>{}, s + 3, par, s1, s0);
    }
    if (ok) {
        // the last plane: its epilogue operands are stage k1's
        const int q = (k1 - kb) & 3;
        const unsigned pq = (unsigned)(((k1 - kb) >> 2) & 1) ^ (q == 3 ? 1u : 0u);
        if (EPI_B && !wait_full(q, pq)) failed = true;
        ok = !__syncthreads_or(failed);
        if (ok && pending) finish(k1 - 1, q);
    }
    if (!ok) {
        // a wait gave up: let the copies already issued land (bounded) before
        // the block's shared memory is released, and record the failure
        if (tid == 0) {
            for (int q = 0; q < 4; ++q)
                if (issued[q] > 0) wait_full(q, (unsigned)(issued[q] - 1) & 1u);  // phases complete in order
            atomicExch(a.err, 1);
        }
        return;
    }
    if (DOT) {
        const double sum = block_sum<NT>(dotv.value(), tid);
        if (tid == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = sum;
    }
}

// Sets the sticky error word (a launch with no kernel able to run it).
__global__ void k_flag_error(int* err) { atomicExch(err, 1); }

// Copies x with the fixed DOFs of the fine level set to 0 (operands supplied by
// a caller may hold values there; the operator ignores them).
__global__ void k_mask_copy(const float* x, const uint8_t* mask, long long nn, float* out) {
    pdl_entry();
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
    int tile;   // 0: 32x8 threads (31x7 nodes), 1: 16x16 threads (15x15 nodes); 2..4 two columns a thread
    int zc;     // node planes per block
    dim3 grid;
};

// Element columns a block covers in x and y (it owns one node fewer each way).
void tile_columns(int tile, int* ex, int* ey) {
    switch (tile) {
        case 0: *ex = 32; *ey = 8; break;
        case kFinePair8x16: *ex = 16; *ey = 16; break;
        case kFinePair16x8: *ex = 32; *ey = 8; break;
        case kFinePair16x16: *ex = 32; *ey = 16; break;
        default: *ex = 16; *ey = 16; break;
    }
}
bool pair_tile(int tile) { return tile >= kFinePair8x16 && tile < kFineTiles; }

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

FinePlan make_plan(int nx, int ny, int nz, int tile, int zc) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    int bx = 0, by = 0;
    tile_columns(tile, &bx, &by);
    const int gx = (NX + bx - 2) / (bx - 1), gy = (NY + by - 2) / (by - 1);
    zc = std::max(1, std::min(zc, NZ));
    return FinePlan{tile, zc, dim3(gx, gy, (NZ + zc - 1) / zc)};
}

// Plans measured by gmg_autotune, per fine grid (process-wide).
std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_plans;

// The cost model: the tile shape and z-chunk length that minimise (waves x
// steps per block) for two resident blocks per SM -- the partial tiles at the
// grid edges and the tail wave are the main losses on grids such as 101^3.
FinePlan model_plan(int nx, int ny, int nz) {
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

// The single-column tile with the same columns, hence the same grid and
// partial count, as `tile`; -1 when there is none.
int single_equivalent(int tile) {
    if (tile == kFinePair8x16) return 1;
    if (tile == kFinePair16x8) return 0;
    return pair_tile(tile) ? -1 : tile;
}

// A tuned plan when gmg_autotune measured one for this grid, else the model's.
FinePlan plan_fine(int nx, int ny, int nz) {
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        const auto it = g_plans.find(std::make_tuple(nx, ny, nz));
        if (it != g_plans.end()) return make_plan(nx, ny, nz, it->second.first, it->second.second);
    }
    return model_plan(nx, ny, nz);
}

template <int MODE, bool DOT>
void launch_shape(const FinePlan& pl, const FineArgs& a, const GSym& G, cudaStream_t s) {
    if (pl.tile == 0) pdl_launch(k_fine<32, 8, MODE, DOT>, dim3(pl.grid), dim3(dim3(32, 8)), 0, s, a, G, pl.zc);
    else pdl_launch(k_fine<16, 16, MODE, DOT>, dim3(pl.grid), dim3(dim3(16, 16)), 0, s, a, G, pl.zc);
}

}  // namespace

int fine_grid_blocks(int nx, int ny, int nz) {
    const FinePlan pl = plan_fine(nx, ny, nz);
    return (int)(pl.grid.x * pl.grid.y * pl.grid.z);
}

int fine_candidates(int nx, int ny, int nz, int max_blocks, int* tiles, int* zcs, int cap) {
    const int NZ = nz + 1;
    int n = 0;
    for (int t = 0; t < kFineTiles; ++t) {
        int last = -1;
        for (int nch = 1; nch <= NZ && n < cap; ++nch) {
            const int zc = (NZ + nch - 1) / nch;
            if (zc < 4 && nch > 1) break;
            if (zc == last) continue;
            last = zc;
            const FinePlan pl = make_plan(nx, ny, nz, t, zc);
            if ((long long)pl.grid.x * pl.grid.y * pl.grid.z > max_blocks) continue;
            tiles[n] = t;
            zcs[n] = zc;
            ++n;
        }
    }
    return n;
}

int fine_plan_blocks(int nx, int ny, int nz, int tile, int zc) {
    const FinePlan pl = make_plan(nx, ny, nz, tile, zc);
    return (int)(pl.grid.x * pl.grid.y * pl.grid.z);
}

void fine_model_plan(int nx, int ny, int nz, int* tile, int* zc) {
    const FinePlan pl = model_plan(nx, ny, nz);
    *tile = pl.tile;
    *zc = pl.zc;
}

void fine_set_plan(int nx, int ny, int nz, int tile, int zc) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const auto key = std::make_tuple(nx, ny, nz);
    if (tile < 0) g_plans.erase(key);
    else g_plans[key] = std::make_pair(tile, zc);
}

void launch_fine(int mode, int dot, int mask_in, const FineArgs& a_in, const GSym& G, cudaStream_t s) {
    // the solver's own level-0 vectors (padded rows, padded moduli): TMA-fed kernel
    if (!mask_in && a_in.Ep && a_in.pitch % 4 == 0 && a_in.pitch > 0 &&
        launch_fine_tma(mode, dot, a_in, G, s) == GMG_OK)
        return;
    // the per-thread-copy kernel runs single-column tiles: the one with the
    // plan's columns (same grid, same partial count), else the model's plan
    FinePlan pl = plan_fine(a_in.nx, a_in.ny, a_in.nz);
    if (single_equivalent(pl.tile) >= 0) {
        pl.tile = single_equivalent(pl.tile);
    } else {
        if (dot && a_in.err) {  // no single-column grid writes this plan's partials
            note_launch();
            k_flag_error<<<1, 1, 0, s>>>(a_in.err);
            return;
        }
        pl = model_plan(a_in.nx, a_in.ny, a_in.nz);
    }
    FineArgs a = a_in;
    if (mask_in && a.scratch) {
        const long long nn = (long long)(a.nx + 1) * (a.ny + 1) * (a.nz + 1);
        note_launch();
        pdl_launch(k_mask_copy, dim3((int)std::min<long long>((3 * nn + 255) / 256, 148 * 8)), dim3(256), 0, s, a.xin, a.mask, nn,
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

namespace {
template <int BX, int BY, int MODE, bool DOT>
int launch_tma_tile(const FinePlan& pl, const FineArgs& a, const GSym& G, cudaStream_t s) {
    using T = TmaTile<BX, BY>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_fine_tma<BX, BY, MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 T::SMEM) != cudaSuccess)
            return GMG_ERR_CUDA;
        attr = true;
    }
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    // node vectors: [NZ][NY][pitch][3] FP32, of which 3 NX floats per row are the grid
    const unsigned long long vd[3] = {3ull * NX, (unsigned long long)NY, (unsigned long long)NZ};
    const unsigned long long vs[2] = {12ull * a.pitch, 12ull * a.pitch * NY};
    const unsigned long long ed[3] = {(unsigned long long)a.nx, (unsigned long long)a.ny, (unsigned long long)a.nz};
    const unsigned long long es[2] = {4ull * a.epitch, 4ull * a.epitch * a.ny};
    const unsigned bx_x[3] = {(unsigned)T::XW, (unsigned)T::XR, 1u};
    const unsigned bx_o[3] = {(unsigned)T::OW, (unsigned)T::OR, 1u};
    const unsigned bx_e[3] = {(unsigned)T::EW, (unsigned)T::ER, 1u};
    CUtensorMap mx, me, mb, md;
    const float* b = a.b ? a.b : a.xin;
    const float* d = a.dold ? a.dold : b;
    if (!encode_f32_map_strided(&mx, a.xin, 3, vd, vs, bx_x) || !encode_f32_map_strided(&me, a.Ep, 3, ed, es, bx_e) ||
        !encode_f32_map_strided(&mb, b, 3, vd, vs, bx_o) || !encode_f32_map_strided(&md, d, 3, vd, vs, bx_o))
        return GMG_ERR_CUDA;
    note_launch();
    pdl_launch(k_fine_tma<BX, BY, MODE, DOT>, dim3(pl.grid), dim3(BX, BY), (size_t)T::SMEM, s, mx, me, mb, md, a, G,
               pl.zc);
    return GMG_OK;
}
template <int MODE, bool DOT>
int launch_tma_shape(const FinePlan& pl, const FineArgs& a, const GSym& G, cudaStream_t s) {
    return pl.tile == 0 ? launch_tma_tile<32, 8, MODE, DOT>(pl, a, G, s) : launch_tma_tile<16, 16, MODE, DOT>(pl, a, G, s);
}
}  // namespace

int launch_fine_tma(int mode, int dot, const FineArgs& a, const GSym& G, cudaStream_t s) {
    if (a.pitch % 4 != 0 || a.epitch % 4 != 0 || !a.Ep) return GMG_ERR_ARG;
    const FinePlan pl = plan_fine(a.nx, a.ny, a.nz);
    if (pair_tile(pl.tile)) return launch_fine_pair(pl.tile, mode, dot, pl.grid, pl.zc, a, G, s);
    if (mode == FM_APPLY) return dot ? launch_tma_shape<FM_APPLY, true>(pl, a, G, s) : launch_tma_shape<FM_APPLY, false>(pl, a, G, s);
    if (mode == FM_SMOOTH)
        return dot ? launch_tma_shape<FM_SMOOTH, true>(pl, a, G, s) : launch_tma_shape<FM_SMOOTH, false>(pl, a, G, s);
    return launch_tma_shape<FM_RESID, false>(pl, a, G, s);
}

bool gsym_from_blocks(const double g[72], GSym* out, double* v64) {
    // value index per entry (class s, row i, column j): 0 a, 1 b (class 0),
    // 2 a', 3 b' (class 7), 4 p, 5 q, 6 c, 7 d, -1 zero
    int which[72];
    for (int t = 0; t < 72; ++t) which[t] = -1;
    auto at = [](int s, int i, int j) { return s * 9 + i * 3 + j; };
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            which[at(0, i, j)] = i == j ? 0 : 1;
            which[at(7, i, j)] = i == j ? 2 : 3;
        }
    const int pair_cls[3] = {1, 2, 4}, pair_rc[3][2] = {{1, 2}, {0, 2}, {0, 1}};
    for (int k = 0; k < 3; ++k) {
        const int s = pair_cls[k], r0 = pair_rc[k][0], r1 = pair_rc[k][1];
        which[at(s, r0, r0)] = which[at(s, r1, r1)] = 4;
        which[at(s, r0, r1)] = which[at(s, r1, r0)] = 5;
    }
    const int c_cls[3] = {3, 5, 6}, c_rc[3][2] = {{0, 1}, {0, 2}, {1, 2}}, d_r[3] = {2, 1, 0};
    for (int k = 0; k < 3; ++k) {
        const int s = c_cls[k], r0 = c_rc[k][0], r1 = c_rc[k][1];
        which[at(s, r0, r0)] = which[at(s, r0, r1)] = which[at(s, r1, r0)] = which[at(s, r1, r1)] = 6;
        which[at(s, d_r[k], d_r[k])] = 7;
    }
    double sum[8] = {}, big = 0.0;
    int cnt[8] = {};
    for (int t = 0; t < 72; ++t) {
        big = std::max(big, std::fabs(g[t]));
        if (which[t] >= 0) {
            sum[which[t]] += g[t];
            ++cnt[which[t]];
        }
    }
    double v[8];
    for (int k = 0; k < 8; ++k) v[k] = sum[k] / cnt[k];
    for (int t = 0; t < 72; ++t)
        if (std::fabs(g[t] - (which[t] >= 0 ? v[which[t]] : 0.0)) > 1e-12 * big) return false;
    out->ab0 = make_float2((float)(v[0] - v[1]), (float)v[1]);
    out->ab7 = make_float2((float)(v[2] - v[3]), (float)v[3]);
    out->pq = make_float2((float)v[4], (float)v[5]);
    out->cd = make_float2((float)v[6], (float)v[7]);
    if (v64) {
        const double w[8] = {v[0] - v[1], v[1], v[2] - v[3], v[3], v[4], v[5], v[6], v[7]};
        for (int k = 0; k < 8; ++k) v64[k] = w[k];
    }
    return true;
}

// Operand B of the tensor-core smoother: row o = the 24 corner forces of an
// element (bottom face corners 00, 10, 01, 11 then the top face, 3 components
// each), column j = the 21 Hadamard modes (monomial m = 1..7, component c:
// j = 3 (m - 1) + c), i.e. G composed with the face split and the corner
// expansion of k_fine, evaluated in FP64 on unit modes.  Stored as BF16 hi and
// lo = bf16(M - hi) in the MMA's K-major core-matrix layout, 32 x 32 each.
static uint16_t host_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
    return (uint16_t)(u >> 16);
}
static float host_bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

void build_tc_operand(const double g[72], uint16_t out[2048]) {
    double M[24][21] = {};
    for (int j = 0; j < 21; ++j) {
        double v[8][3] = {}, w[8][3] = {};
        v[1 + j / 3][j % 3] = 1.0;
        for (int sg = 0; sg < 8; ++sg)
            for (int i = 0; i < 3; ++i) {
                const int mi = mono(sg, i);
                if (mi == 0) continue;
                double acc = 0.0;
                for (int jj = 0; jj < 3; ++jj) {
                    const int mj = mono(sg, jj);
                    if (mj == 0) continue;
                    acc += g[sg * 9 + i * 3 + jj] * v[mj][jj];
                }
                w[mi][i] = acc;
            }
        for (int f = 0; f < 2; ++f)
            for (int c = 0; c < 3; ++c) {
                double S[4];
                for (int q = 0; q < 4; ++q) S[q] = f == 0 ? w[q][c] - w[q + 4][c] : w[q][c] + w[q + 4][c];
                const double pp = S[0] - S[2], qd = S[1] - S[3], r = S[0] + S[2], sd = S[1] + S[3];
                const double corner[4] = {pp - qd, pp + qd, r - sd, r + sd};
                for (int q = 0; q < 4; ++q) M[f * 12 + q * 3 + c][j] = corner[q];
            }
    }
    std::memset(out, 0, 2048 * sizeof(uint16_t));
    for (int o = 0; o < 24; ++o)
        for (int j = 0; j < 21; ++j) {
            const int idx = ((o >> 3) * 4 + (j >> 3)) * 64 + (o & 7) * 8 + (j & 7);
            const uint16_t hi = host_bf16((float)M[o][j]);
            out[idx] = hi;
            out[1024 + idx] = host_bf16((float)(M[o][j] - (double)host_bf16_value(hi)));
        }
}

namespace {
template <int BX, int BY, int PASSES, bool DOT>
void launch_tc_tile(const FinePlan& pl, const FineArgs& a, cudaStream_t s) {
    constexpr int dyn = (PASSES > 1 ? 2 : 1) * 2 * kTcTileBytes + 4096;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_fine_tc<BX, BY, PASSES, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        attr = true;
    }
    k_fine_tc<BX, BY, PASSES, DOT><<<pl.grid, dim3(BX, BY), dyn, s>>>(a, pl.zc);
}
template <int PASSES, bool DOT>
void launch_tc_shape(const FinePlan& pl, const FineArgs& a, cudaStream_t s) {
    if (pl.tile == 0) launch_tc_tile<32, 8, PASSES, DOT>(pl, a, s);
    else launch_tc_tile<16, 16, PASSES, DOT>(pl, a, s);
}
}  // namespace

void launch_fine_tc(int passes, int dot, const FineArgs& a, cudaStream_t s) {
    const FinePlan pl = plan_fine(a.nx, a.ny, a.nz);
    note_launch();
    if (passes > 1) {
        if (dot) launch_tc_shape<3, true>(pl, a, s);
        else launch_tc_shape<3, false>(pl, a, s);
    } else {
        if (dot) launch_tc_shape<1, true>(pl, a, s);
        else launch_tc_shape<1, false>(pl, a, s);
    }
}

void launch_hadamard_blocks(const double* Ke, double* g72, cudaStream_t s) {
    note_launch();
    k_hadamard_blocks<<<1, 96, 0, s>>>(Ke, g72);
}

}  // namespace gmg
