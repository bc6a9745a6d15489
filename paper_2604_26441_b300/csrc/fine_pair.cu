// Matrix-free fine-level operator (Eq. mf_matvec) with two element columns per
// thread, for sm_103a.
//
// The arithmetic is the Walsh-Hadamard form of the single-column operator in
// fine.cu (K_e = H^T G H with eight 3x3 parity blocks taking eight distinct
// values; per element 21 mode sums and the symmetric contraction of G),
// the same operations in the same order, so that every output is bitwise equal
// to that kernel's.  What changes is the unit of work of a thread:
//   - thread (tx, ty) holds the two x-adjacent element columns whose low corners
//     are nodes (x0-1+2tx, y0-1+ty) and (x0+2tx, y0-1+ty), and owns the nodes
//     x0+2tx (between its columns) and x0+2tx+1 (between its second column and
//     the next thread's first);
//   - every value is carried as f32x2 pairs whose two lanes are the two columns
//     (x, y and z components each a pair), so each add, subtract, FMA and
//     product of the element arithmetic is one packed instruction (FADD2,
//     FFMA2, FMUL2) for two elements, and the eight coefficients, scaled by
//     each column's modulus, form one pair per coefficient;
//   - the wait, barrier, mask, index and shuffle work of a layer is paid once
//     per two elements, and the sum across the shared node of the two columns
//     stays in registers (one shuffle per component reaches the next thread).
// A block of BX x BY threads covers 2BX x BY element columns and owns
// (2BX-1) x (BY-1) nodes.  Staging is that of the single-column TMA kernel: per
// z-step one thread issues the node plane, the moduli layer and the epilogue
// operands as 3D tensor boxes into a 4-slot shared-memory ring on one mbarrier
// per slot, three steps ahead; waits are bounded, and a block that gives up
// waits (bounded) for its own copies in flight and sets the sticky error word.
#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace gmg {

namespace {

__host__ __device__ constexpr int pround4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int pround128(int v) { return (v + 127) / 128 * 128; }
__device__ __forceinline__ int pfloor4(int v) { return v & ~3; }

// A node or element quantity of the two columns: lane .x is the first column,
// lane .y the second.  a - b is formed as fma(b, -1, a), which rounds exactly
// like the subtraction.
struct P3 {
    float2 x, y, z;
};
__device__ __forceinline__ P3 padd(const P3& a, const P3& b) {
    return {__fadd2_rn(a.x, b.x), __fadd2_rn(a.y, b.y), __fadd2_rn(a.z, b.z)};
}
__device__ __forceinline__ P3 psub(const P3& a, const P3& b) {
    const float2 m = make_float2(-1.f, -1.f);
    return {__ffma2_rn(b.x, m, a.x), __ffma2_rn(b.y, m, a.y), __ffma2_rn(b.z, m, a.z)};
}
__device__ __forceinline__ float2 pcomp(const P3& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }
__device__ __forceinline__ P3 pzero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// Difference sums of the four corners of a face (x fastest): q[1] = x-difference,
// q[2] = y-difference, q[3] = xy-difference.
__device__ __forceinline__ void pface(const P3 c[4], P3 q[4]) {
    const P3 dx0 = psub(c[1], c[0]), dx1 = psub(c[3], c[2]);
    q[1] = padd(dx0, dx1);
    q[2] = padd(psub(c[2], c[0]), psub(c[3], c[1]));
    q[3] = psub(dx1, dx0);
}

// Layer state carried along z: corners and face differences of the shared face,
// the top-face quantities of the layer and the two columns' moduli.
struct PLayer {
    P3 C[4];
    P3 Q[4];  // Q[0] unused
    P3 T[4];
    float2 E;
};

// Shared-memory layout of one block: a 4-slot ring of stages (node plane, moduli
// layer, right-hand side and previous increment of the plane being finished),
// the y-exchange of the node sums and the ring's mbarriers.
template <int BX, int BY>
struct PairTile {
    static constexpr int EX = 2 * BX;                     // element columns per row
    static constexpr int XW = pround4(3 * (EX + 1) + 3);  // floats per staged node row (+ up to 3 of offset)
    static constexpr int XR = BY + 1;                     // node rows
    static constexpr int EW = pround4(EX + 3);            // moduli per staged row
    static constexpr int ER = BY;
    static constexpr int OW = pround4(3 * (EX - 1) + 3);  // floats per row of owned nodes
    static constexpr int OR = BY - 1;
    static constexpr int XB = XW * XR * 4, EB = EW * ER * 4, OB = OW * OR * 4;
    static constexpr int XOFF = 0;
    static constexpr int EOFF = pround128(XB);
    static constexpr int BOFF = EOFF + pround128(EB);
    static constexpr int DOFF = BOFF + pround128(OB);
    static constexpr int STAGE = DOFF + pround128(OB);
    // y-exchange: [2][BY + 1][BX] records of 8 floats (x, y, z and modulus sum,
    // each a pair over the thread's two nodes); row BY is never written
    static constexpr int SXOFF = 4 * STAGE;
    static constexpr int BAROFF = SXOFF + 2 * (BY + 1) * BX * 32;
    static constexpr int SMEM = BAROFF + 4 * 8;
};

constexpr unsigned kPairSpin = 1u << 22;

}  // namespace

namespace {

template <int NTH>
__device__ __forceinline__ double pblock_sum(double v, int tid) {
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

// ~210 registers a thread: two 128-thread blocks or one 256-thread block per SM
template <int BX, int BY, int MODE, bool DOT>
__global__ void __launch_bounds__(BX * BY, BX * BY >= 256 ? 1 : 2)
k_fine_pair(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tme,
            const __grid_constant__ CUtensorMap tmb, const __grid_constant__ CUtensorMap tmd, FineArgs a,
            const __grid_constant__ GSym G, int zchunk) {
    using T = PairTile<BX, BY>;
    constexpr int NT = BX * BY;
    constexpr bool EPI_B = MODE != FM_APPLY;
    constexpr bool EPI_D = MODE == FM_SMOOTH;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    float4(*sx)[BY + 1][BX][2] = reinterpret_cast<float4(*)[BY + 1][BX][2]>(smem + T::SXOFF);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + T::BAROFF);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int px = a.pitch, NXYp = px * NY;
    [[maybe_unused]] const long long nvec = (long long)NXYp * NZ;  // bounds of the checked build
    const int x0 = blockIdx.x * (2 * BX - 1), y0 = blockIdx.y * (BY - 1);
    const int k0 = blockIdx.z * zchunk, k1 = min(k0 + zchunk, NZ);
    const int kb = k0 - 1;
    // box origins (innermost coordinate rounded down to 4 floats) and offsets
    const int xs = pfloor4(3 * (x0 - 1)), es = pfloor4(x0 - 1), bs = pfloor4(3 * x0);
    const int rx = ty * T::XW + 6 * tx + (3 * (x0 - 1) - xs);  // first column's low corner in a node plane
    const int re = ty * T::EW + 2 * tx + (x0 - 1 - es);        // first column's modulus in a layer
    const int rb = ty * T::OW + 6 * tx + (3 * x0 - bs);        // first owned node in an epilogue plane
    const int oxa = x0 + 2 * tx, oy = y0 + ty;
    const bool own_a = ty < BY - 1 && oy < NY && oxa < NX;
    const bool own_b = own_a && tx < BX - 1 && oxa + 1 < NX;
    const int onode = oy * px + oxa;
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
    // operands may only be read after the previous kernel of the stream is done
    pdl_entry();

    // stage s into its ring slot (thread 0 only); issued[q] counts the phases
    // started on slot q, for the failure path
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
        for (unsigned it = 0; it < kPairSpin; ++it)
            if (mbar_try_wait(&full[q], parity)) return true;
        return false;
    };
    // the two owned nodes' masks as one int (bits 0-2 node a, 3-5 node b);
    // nodes a thread does not own read as all fixed
    auto load_mask = [&](int kp) -> int {
        const bool in = kp >= k0 && kp < k1;
        const int ma = (own_a && in) ? (int)a.mask[GMG_B(onode + kp * NXYp, nvec, 121)] : 7;
        const int mb = (own_b && in) ? (int)a.mask[GMG_B(onode + 1 + kp * NXYp, nvec, 122)] : 7;
        return ma | (mb << 3);
    };
    // the three nodes of rows y and y+1 that the two columns touch, as the four
    // corner pairs (x-,y-), (x+,y-), (x-,y+), (x+,y+), and their differences
    auto load_plane = [&](const float* p, PLayer& L) {
        const float* p1 = p + T::XW;
        L.C[0] = {make_float2(p[0], p[3]), make_float2(p[1], p[4]), make_float2(p[2], p[5])};
        L.C[1] = {make_float2(p[3], p[6]), make_float2(p[4], p[7]), make_float2(p[5], p[8])};
        L.C[2] = {make_float2(p1[0], p1[3]), make_float2(p1[1], p1[4]), make_float2(p1[2], p1[5])};
        L.C[3] = {make_float2(p1[3], p1[6]), make_float2(p1[4], p1[7]), make_float2(p1[5], p1[8])};
        pface(L.C, L.Q);
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
    PLayer s0, s1;
    load_plane(reinterpret_cast<const float*>(smem + 3 * T::STAGE + T::XOFF) + rx, s0);
#pragma unroll
    for (int q = 0; q < 4; ++q) s0.T[q] = pzero();
    s0.E = make_float2(0.f, 0.f);
    // masks four planes ahead, one register per ring slot (the slot of step s
    // holds plane s's masks), so a load's result is not touched before its use
    int mq[4] = {7 | (7 << 3), load_mask(k0), load_mask(k0 + 1), load_mask(k0 + 2)};
    bool pending = false;
    P3 R1 = pzero(), un_pend = pzero();
    float2 eR1 = make_float2(0.f, 0.f);
    int m_pend = 7 | (7 << 3);
    DSAcc dotv;

    // Epilogue of the two owned nodes of plane kp from the stage in slot q,
    // branch-free (unowned nodes hold an all-fixed mask; only stores are
    // predicated).  Lane .x of every pair is node a, lane .y node b.
    auto finish = [&](int kp, int q) {
        const float4 u0 = sx[kp & 1][ty + 1][tx][0], u1 = sx[kp & 1][ty + 1][tx][1];
        const P3 y = padd(R1, P3{make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y)});
        const long long on = own_a ? GMG_B(onode + kp * NXYp, nvec, 123) : 0;
        const long long onb = own_b ? GMG_B(onode + 1 + kp * NXYp, nvec, 124) : 0;
        float* out = a.out;
        bool fa[3], fb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fa[c] = !((m_pend >> c) & 1);
            fb[c] = !((m_pend >> (3 + c)) & 1);
        }
        if (MODE == FM_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 yc = pcomp(y, c), uc = pcomp(un_pend, c);
                const float va = fa[c] ? yc.x : 0.f, vb = fb[c] ? yc.y : 0.f;
                if (own_a) out[3 * on + c] = va;
                if (own_b) out[3 * onb + c] = vb;
                if (DOT) {
                    dotv.add_prod(fa[c] ? uc.x : 0.f, va);
                    dotv.add_prod(fb[c] ? uc.y : 0.f, vb);
                }
            }
        } else {
            const float* bb = reinterpret_cast<const float*>(smem + q * T::STAGE + T::BOFF) + rb;
            const float2 m1 = make_float2(-1.f, -1.f);
            if (MODE == FM_RESID) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 r = __ffma2_rn(pcomp(y, c), m1, make_float2(bb[c], bb[3 + c]));
                    if (own_a) out[3 * on + c] = fa[c] ? r.x : 0.f;
                    if (own_b) out[3 * onb + c] = fb[c] ? r.y : 0.f;
                }
            } else {
                const float* dd = reinterpret_cast<const float*>(smem + q * T::STAGE + T::DOFF) + rb;
                const float2 den = __fmul2_rn(make_float2(a.kd, a.kd), __fadd2_rn(eR1, make_float2(u1.z, u1.w)));
                const float2 cai = __fmul2_rn(make_float2(ca, ca), make_float2(jacobi_rcp(den.x), jacobi_rcp(den.y)));
                float* dn_out = a.dnew;
                const bool wa = own_a && dn_out != nullptr, wb = own_b && dn_out != nullptr;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float2 d = __fmul2_rn(cai, __ffma2_rn(pcomp(y, c), m1, make_float2(bb[c], bb[3 + c])));
                    if (need_d) d = __ffma2_rn(make_float2(cd, cd), make_float2(dd[c], dd[3 + c]), d);
                    d = make_float2(fa[c] ? d.x : 0.f, fb[c] ? d.y : 0.f);
                    const float2 xs2 = __fadd2_rn(pcomp(un_pend, c), d);
                    const float xa = fa[c] ? xs2.x : 0.f, xb = fb[c] ? xs2.y : 0.f;
                    if (DOT) {
                        dotv.add_prod(fa[c] ? bb[c] : 0.f, xa);
                        dotv.add_prod(fb[c] ? bb[3 + c] : 0.f, xb);
                    }
                    if (own_a) out[3 * on + c] = xa;
                    if (own_b) out[3 * onb + c] = xb;
                    if (wa) dn_out[3 * on + c] = d.x;
                    if (wb) dn_out[3 * onb + c] = d.y;
                }
            }
        }
    };

    // one step s = one element layer (bottom face in `in`, top face into `out`)
    // with the stage in slot Q; `par` is the trip's phase bit
    auto step = [&](auto Qc, const int s, const unsigned par, const PLayer& in, PLayer& out) -> bool {
        constexpr int Q = decltype(Qc)::value;
        if (!wait_full(Q, par ^ (Q == 3 ? 1u : 0u))) failed = true;
        if (__syncthreads_or(failed)) return false;
        if (tid == 0 && s + 3 <= k1) issue(s + 3);
        if (pending) finish(s - 1, Q);
        pending = false;
        const int mcur = mq[Q];
        mq[Q] = load_mask(s + 4);
        load_plane(reinterpret_cast<const float*>(smem + Q * T::STAGE + T::XOFF) + rx, out);
        {
            const float* pe = reinterpret_cast<const float*>(smem + Q * T::STAGE + T::EOFF) + re;
            out.E = make_float2(pe[0], pe[1]);
        }
        P3 v[8];
        {
            const P3 z00 = psub(out.C[0], in.C[0]), z10 = psub(out.C[1], in.C[1]);
            const P3 z01 = psub(out.C[2], in.C[2]), z11 = psub(out.C[3], in.C[3]);
            v[4] = padd(padd(z00, z10), padd(z01, z11));
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                v[q] = padd(out.Q[q], in.Q[q]);
                v[q + 4] = psub(out.Q[q], in.Q[q]);
            }
        }
        P3 w[8];
        w[0] = pzero();
        {
            float2 u[8][3], o[8][3];
#pragma unroll
            for (int m = 1; m < 8; ++m) {
                u[m][0] = v[m].x;
                u[m][1] = v[m].y;
                u[m][2] = v[m].z;
            }
            gsym_contract(gsym_scale2(G, out.E), u, o);
#pragma unroll
            for (int m = 1; m < 8; ++m) w[m] = P3{o[m][0], o[m][1], o[m][2]};
        }
        P3 Bf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out.T[q] = padd(w[q], w[q + 4]);
            Bf[q] = psub(w[q], w[q + 4]);
        }
        if (s >= k0) {
            const P3 S0 = padd(in.T[0], Bf[0]), S1 = padd(in.T[1], Bf[1]);
            const P3 S2 = padd(in.T[2], Bf[2]), S3 = padd(in.T[3], Bf[3]);
            const P3 p = psub(S0, S2), qd = psub(S1, S3), r = padd(S0, S2), sd = padd(S1, S3);
            const P3 c00 = psub(p, qd), c10 = padd(p, qd), c01 = psub(r, sd), c11 = padd(r, sd);
            // the x- corners to the right of the two owned nodes: the second
            // column's, and the next thread's first column's
            const P3 n01{make_float2(c01.x.y, __shfl_down_sync(FULL, c01.x.x, 1, BX)),
                         make_float2(c01.y.y, __shfl_down_sync(FULL, c01.y.x, 1, BX)),
                         make_float2(c01.z.y, __shfl_down_sync(FULL, c01.z.x, 1, BX))};
            const P3 n00{make_float2(c00.x.y, __shfl_down_sync(FULL, c00.x.x, 1, BX)),
                         make_float2(c00.y.y, __shfl_down_sync(FULL, c00.y.x, 1, BX)),
                         make_float2(c00.z.y, __shfl_down_sync(FULL, c00.z.x, 1, BX))};
            R1 = padd(c11, n01);
            const P3 r0 = padd(c10, n00);
            const float2 esum = __fadd2_rn(in.E, out.E);
            const float2 er = __fadd2_rn(esum, make_float2(esum.y, __shfl_down_sync(FULL, esum.x, 1, BX)));
            sx[s & 1][ty][tx][0] = make_float4(r0.x.x, r0.x.y, r0.y.x, r0.y.y);
            sx[s & 1][ty][tx][1] = make_float4(r0.z.x, r0.z.y, er.x, er.y);
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
        const double sum = pblock_sum<NT>(dotv.value(), tid);
        if (tid == 0) a.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = sum;
    }
}

}  // namespace

namespace {

template <int BX, int BY, int MODE, bool DOT>
int launch_pair_tile(dim3 grid, int zc, const FineArgs& a, const GSym& G, cudaStream_t s) {
    using T = PairTile<BX, BY>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_fine_pair<BX, BY, MODE, DOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    pdl_launch(k_fine_pair<BX, BY, MODE, DOT>, grid, dim3(BX, BY), (size_t)T::SMEM, s, mx, me, mb, md, a, G, zc);
    return GMG_OK;
}

template <int MODE, bool DOT>
int launch_pair_shape(int tile, dim3 grid, int zc, const FineArgs& a, const GSym& G, cudaStream_t s) {
    switch (tile) {
        case kFinePair8x16: return launch_pair_tile<8, 16, MODE, DOT>(grid, zc, a, G, s);
        case kFinePair16x8: return launch_pair_tile<16, 8, MODE, DOT>(grid, zc, a, G, s);
        case kFinePair16x16: return launch_pair_tile<16, 16, MODE, DOT>(grid, zc, a, G, s);
        default: return GMG_ERR_ARG;
    }
}

}  // namespace

int launch_fine_pair(int tile, int mode, int dot, dim3 grid, int zc, const FineArgs& a, const GSym& G,
                     cudaStream_t s) {
    if (a.pitch % 4 != 0 || a.epitch % 4 != 0 || !a.Ep) return GMG_ERR_ARG;
    if (mode == FM_APPLY)
        return dot ? launch_pair_shape<FM_APPLY, true>(tile, grid, zc, a, G, s)
                   : launch_pair_shape<FM_APPLY, false>(tile, grid, zc, a, G, s);
    if (mode == FM_SMOOTH)
        return dot ? launch_pair_shape<FM_SMOOTH, true>(tile, grid, zc, a, G, s)
                   : launch_pair_shape<FM_SMOOTH, false>(tile, grid, zc, a, G, s);
    return launch_pair_shape<FM_RESID, false>(tile, grid, zc, a, G, s);
}

}  // namespace gmg
