// Tensor-core level-0 operator of the multi-load path: y = K u (Eq. mf_matvec)
// for 8 loads per CTA as a dense element contraction on tcgen05 (kind::tf32,
// FP32 accumulation in TMEM), fused with the apply / residual / smoother
// epilogues of the CUDA-core operator.
//
// Contraction.  For every element e and load l the 24 corner forces are
// f(e,l) = E_e K_e u(e,l).  One MMA tile is M = 128 rows = 16 x-consecutive
// elements x 8 loads, N = 32 columns (the 24 forces, corner a = dx + 2 dy +
// 4 dz, component c: column 3a + c; 8 zero columns), and K runs over the 8
// corners x (x, y, z, pad) of the element.  The staged node planes hold the
// loads' 16-byte records (x, y, z, 0), a node's 8 loads in 128 contiguous bytes,
// so the 8 rows of one core matrix are the 8 loads of one element's corner and
// the A operand of corner pair (dx = 0, 1; dy, dz) is the staged plane seen
// through a shifted descriptor: no operand is packed by threads.  Four MMAs
// (dy, dz) of K = 8 cover the element.
//
// Precision.  TF32 keeps 11 significant bits, so u enters as three TF32 limbs
// on a block-floating-point grid per plane and load (hi: 11 bits of the
// plane's largest magnitude, mid: the next 11, lo: the rest): u = hi + mid +
// lo, exactly where |u| is within 2^-12 of the plane's largest value.  K_e enters as an integer matrix
// times a scale when it is one (for nu = 0.3 the entries are integers up to 88
// times one constant, exact in TF32): three MMAs per corner pair, every product
// exact.  The MMAs run limb-major (the four corner pairs of hi, then of mid,
// then of lo): the operator is applied to smooth fields (PCG directions,
// smoother iterates) whose image K u is many orders smaller than |K| |u|, and
// in this order every running sum stays a whole number of the current limb's
// quantum below 2^24 quanta -- the hi sum is exact, and once all corners are in
// it has cancelled down to |K| |u - hi|, so the mid and lo sums are exact too.
// (Corner-pair-major order, two limbs, or limbs rounded per value -- whose
// quanta differ wherever u changes sign -- left errors of 1e-5 to 1e-3 of K u
// for the smoothest fields and cost PCG iterations.)  When K_e is not such a multiple it is split
// into hi + lo as well and two more MMAs add hi(u) lo(K_e), mid(u) lo(K_e).
// E_e and the scale multiply the forces in FP32.
//
// Schedule.  A CTA (16 warps, one per SM: 203 KB of shared memory, all 512
// TMEM columns) owns 15 x 7 nodes of a plane and marches along z through a
// chunk of planes; it computes the 16 x 8 elements around them (a one-element
// halo).  Node planes arrive by TMA into a ring of three slots with the moduli
// of the layer below; all threads split each plane into its limbs.  One thread
// issues the 8 tiles x 12 (or 20) MMAs of layer z into one half of TMEM while
// the others read layer z-1's forces from the other half (tcgen05.ld), scale
// them by E_e, add the top-face forces kept from layer z-2 and sum each node's
// four cells in shared memory in four parity passes (no atomics: each pass
// writes every node at most once, in a fixed order), then run the epilogue of
// plane z-1 for the owned nodes.  Every wait is bounded; a wait that gives up
// sets the error word and the CTA drains its copies and MMAs before it exits.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace gmg {

namespace {

constexpr int kTEX = 16, kTEY = 8;                    // elements of a tile: x, y (= MMA tiles per layer)
constexpr int kTNX = kTEX + 1, kTNY = kTEY + 1;       // staged nodes
constexpr int kOwnX = kTEX - 1, kOwnY = kTEY - 1;     // owned nodes
constexpr int kLG = 8;                                // loads per CTA
constexpr int kNodeB = kLG * 16;                      // bytes per staged node
constexpr int kRowB = kTNX * kNodeB;                  // bytes per staged node row
constexpr int kPlaneB = kTNY * kRowB;                 // bytes per staged plane (one limb)
constexpr int kPlaneRec = kTNX * kTNY * kLG;          // records per staged plane
constexpr int kEW = 20;                               // moduli per staged row (16 + offset, rounded to 4)
constexpr int kEB = kEW * kTEY * 4;
constexpr int kLimbs = 3;                             // TF32 limbs of u: hi, mid, lo
constexpr int kSlotB = (kLimbs * kPlaneB + kEB + 127) / 128 * 128;  // limbs, moduli
constexpr int kNFOff = 3 * kSlotB;                    // node-force plane [9][17][8] float4
constexpr int kBOff = kNFOff + kPlaneB;               // K_e operand, 2 limbs x 4 KB
constexpr int kBarOff = kBOff + 8192;
constexpr int kRedOff = kBarOff + 64;
constexpr int kSmemUsed = kRedOff + 16 * kLG * 8;
constexpr int kSmem = kSmemUsed + 1024;               // slack for the 1 KB alignment of the base
constexpr int kTcThreads = 512;
constexpr unsigned kTcSpinM = 1u << 22;
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

static_assert(kSmem <= 227 * 1024, "one CTA per SM");
static_assert(kSlotB % 128 == 0 && kPlaneB % 128 == 0 && kNFOff % 128 == 0 && kBOff % 128 == 0, "TMA alignment");

__device__ __forceinline__ bool fbit(uint8_t m, int c) { return (m >> c) & 1; }

__device__ __forceinline__ uint64_t mdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    // K-major, no swizzle: lbo = byte distance of K-adjacent core matrices,
    // sbo = byte distance of adjacent 8-row groups
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_tf32_m(unsigned d, uint64_t da, uint64_t db, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
          "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
          "r"(smem_u32(bar))
        : "memory");
}

// 24 columns of this warp's TMEM lane quarter: x16 + x8.
__device__ __forceinline__ void tmem_ld24(unsigned addr, float* v) {
    unsigned r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                   "=r"(r[23])
                 : "r"(addr + 16u));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}

template <int MODE, bool DOT, int PASSES>
__global__ void __launch_bounds__(kTcThreads, 1)
k_mfine_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tme, MFineArgs a,
           const float* __restrict__ Bop, float scale, int zchunk, int gx, int gy, int ngroups) {
    extern __shared__ unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    uint64_t* tbar = reinterpret_cast<uint64_t*>(sm + kBarOff);  // [3] plane slots
    uint64_t* mbar = tbar + 3;                                   // [2] TMEM halves
    unsigned* tslot = reinterpret_cast<unsigned*>(mbar + 2);
    double* red = reinterpret_cast<double*>(sm + kRedOff);
    float4* NF = reinterpret_cast<float4*>(sm + kNFOff);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2;                 // TMEM lane quarter, warpgroup (tiles 2g, 2g+1)
    const int e = 4 * q + (lane >> 3), l = lane & 7;       // this thread's element (x) and load in a tile
    const int lg = (int)(blockIdx.x % (unsigned)ngroups);
    const int tile = (int)(blockIdx.x / (unsigned)ngroups);
    const int txi = tile % gx, tyi = (tile / gx) % gy, tzi = tile / (gx * gy);
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const int x0e = kOwnX * txi - 1, y0e = kOwnY * tyi - 1;  // first element of the tile
    const int k0 = tzi * zchunk, k1 = min(k0 + zchunk, NZ), kb = k0 - 1;
    const int es = x0e & ~3, xoff = x0e - es;                // moduli box origin (rounded down to 4)
    const float cd = MODE == FM_SMOOTH ? (float)a.coef[2 * a.step] : 0.f;
    const float ca = MODE == FM_SMOOTH ? (float)a.coef[2 * a.step + 1] : 0.f;

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(&tbar[i], 1);
        for (int i = 0; i < 2; ++i) mbar_init(&mbar[i], 1);
        mbar_fence_init();
    }
    pdl_entry();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(Bop);
        uint4* dst = reinterpret_cast<uint4*>(sm + kBOff);
        for (int i = tid; i < 8192 / 16; i += kTcThreads) dst[i] = src[i];
        for (int i = tid; i < kPlaneRec; i += kTcThreads) NF[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;

    // for the drain (thread 0's view): the last plane issued and the last one
    // waited for, the last layer whose MMAs were committed and the last one
    // waited for; copies and commits complete in order on each barrier
    int p_iss = kb - 1, p_con = kb - 1, z_iss = kb - 1, z_con = kb - 1;
    auto slot_of = [&](int p) { return (p - kb) % 3; };
    auto issue_plane = [&](int p) {  // node plane p and moduli layer p - 1
        const int s = slot_of(p);
        unsigned char* st = sm + s * kSlotB;
        mbar_expect_tx(&tbar[s], (unsigned)(kPlaneB + kEB));
        tma4(st, &tmx, 32 * lg, x0e, y0e, p, &tbar[s]);
        tma3(st + kLimbs * kPlaneB, &tme, es, y0e, p - 1, &tbar[s]);
        p_iss = p;
    };
    auto wait_bar = [&](uint64_t* bar, unsigned parity) -> bool {
        for (unsigned it = 0; it < kTcSpinM; ++it)
            if (mbar_try_wait(bar, parity)) return true;
        return false;
    };
    // a phase counts as consumed only when its wait succeeded (the drain waits
    // again for the others)
    auto wait_plane = [&](int p) -> bool {
        const int s = slot_of(p);
        const bool ok = wait_bar(&tbar[s], (unsigned)(((p - kb) / 3) & 1));
        if (ok) p_con = p;
        return ok;
    };
    auto wait_mma = [&](int z) -> bool {
        const int b = (z - kb) & 1;
        const bool ok = wait_bar(&mbar[b], (unsigned)(((z - kb) >> 1) & 1));
        if (ok) z_con = z;
        return ok;
    };
    // The record (in the hi limb) -> hi, mid, lo on a grid shared by the whole
    // plane of each load: Q = 2^(E - 10) with 2^E the plane's largest |u|
    // component for that load (block floating point), hi = Q rint(u / Q),
    // mid = (Q / 2^11) rint((u - hi) / (Q / 2^11)), lo the rest.  Every limb is
    // a TF32 number; all hi products of an element are multiples of one or two
    // neighbouring quanta, so their sum is exact even where u changes sign or
    // magnitude inside the element, and mid and lo follow at 2^-11 and 2^-22.
    float* const qred = reinterpret_cast<float*>(red);  // [16 warps][8 loads] maxima (scratch shared with the dot sums)
    auto split = [&](int p) {
        unsigned char* st = sm + slot_of(p) * kSlotB;
        float4* hi = reinterpret_cast<float4*>(st);
        float4* mid = reinterpret_cast<float4*>(st + kPlaneB);
        float4* lo = reinterpret_cast<float4*>(st + 2 * kPlaneB);
        float mx = 0.f;  // this thread's records all belong to load tid % 8
        for (int r = tid; r < kPlaneRec; r += kTcThreads) {
            const float4 v = hi[r];
            mx = fmaxf(mx, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
        __syncthreads();  // the previous split's reads of qred are done
        if (lane < kLG) qred[warp * kLG + lane] = mx;
        __syncthreads();
        float m = 0.f;
#pragma unroll
        for (int w = 0; w < 16; ++w) m = fmaxf(m, qred[w * kLG + (tid & 7)]);
        int ex = 0;
        (void)frexpf(m, &ex);                  // m < 2^ex (m = 0: ex = 0)
        const float Q = ldexpf(1.f, ex - 11), iQ = ldexpf(1.f, 11 - ex);
        const float Qm = ldexpf(1.f, ex - 22), iQm = ldexpf(1.f, 22 - ex);
        for (int r = tid; r < kPlaneRec; r += kTcThreads) {
            const float4 v = hi[r];
            const float4 h = make_float4(rintf(v.x * iQ) * Q, rintf(v.y * iQ) * Q, rintf(v.z * iQ) * Q, 0.f);
            const float4 r1 = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, 0.f);  // exact
            const float4 mm = make_float4(rintf(r1.x * iQm) * Qm, rintf(r1.y * iQm) * Qm, rintf(r1.z * iQm) * Qm, 0.f);
            hi[r] = h;
            mid[r] = mm;
            lo[r] = make_float4(r1.x - mm.x, r1.y - mm.y, r1.z - mm.z, 0.f);  // exact
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    auto issue_mma = [&](int z) {  // layer z (planes z, z + 1) into TMEM half (z - kb) & 1
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int b = (z - kb) & 1;
        const unsigned p0 = smem_u32(sm + slot_of(z) * kSlotB), p1 = smem_u32(sm + slot_of(z + 1) * kSlotB);
        const unsigned bb = smem_u32(sm + kBOff);
        // limb-major: all hi products of the element first (their running sum
        // is exact: one quantum, far from 2^24 quanta), then mid, then lo.
        // Descriptors: the plane and operand bases once, then compile-time
        // offsets (the address field holds byte address / 16 in its low bits).
        const uint64_t dA0 = mdesc(p0, kNodeB, kNodeB), dA1 = mdesc(p1, kNodeB, kNodeB), dB = mdesc(bb, 512, 128);
#pragma unroll
        for (int t = 0; t < kTEY; ++t) {
            const unsigned d = tmem + (unsigned)(b * 256 + t * 32);
#pragma unroll
            for (int pass = 0; pass < PASSES; ++pass) {
                const int limb = pass < 3 ? pass : pass - 3;  // u limb: hi, mid, lo (then hi, mid with K_e lo)
                const unsigned boff = pass < 3 ? 0u : 4096u;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int dy = j & 1, dz = j >> 1;
                    const uint64_t da = (dz ? dA1 : dA0) + (uint64_t)(((t + dy) * kRowB + limb * kPlaneB) >> 4);
                    const uint64_t db = dB + (uint64_t)((boff + (unsigned)(j * 1024)) >> 4);
                    mma_tf32_m(d, da, db, (pass > 0 || j > 0) ? 1u : 0u);
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar[b]))
                     : "memory");
        z_iss = z;
    };

    float top[2][12];
#pragma unroll
    for (int tt = 0; tt < 2; ++tt)
#pragma unroll
        for (int i = 0; i < 12; ++i) top[tt][i] = 0.f;
    DSAcc dotv;

    // forces of layer zz (TMEM half (zz - kb) & 1) -> node sums of plane zz ->
    // its epilogue (plane zz owned: zz >= k0)
    auto process = [&](int zz) {
        const int bz = (zz - kb) & 1;
        const float* sE = reinterpret_cast<const float*>(sm + slot_of(zz + 1) * kSlotB + kLimbs * kPlaneB);
        float bot[2][12];
#pragma unroll
        for (int tt = 0; tt < 2; ++tt) {
            const int t = 2 * g + tt;
            float f[24];
            tmem_ld24(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(bz * 256 + t * 32), f);
            const float Es = sE[t * kEW + e + xoff] * scale;
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                bot[tt][i] = fmaf(f[i], Es, top[tt][i]);
                top[tt][i] = f[12 + i] * Es;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (zz < k0) return;
        // the four cells around each node, four parity passes (px, py)
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int px = pass & 1, py = pass >> 1;
            if ((e & 1) == px) {
                const int t = 2 * g + py;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int dx = c4 & 1, dy = c4 >> 1;
                    float4* nf = &NF[((t + dy) * kTNX + (e + dx)) * kLG + l];
                    float4 v = *nf;
                    v.x += bot[py][3 * c4];
                    v.y += bot[py][3 * c4 + 1];
                    v.z += bot[py][3 * c4 + 2];
                    *nf = v;
                }
            }
            __syncthreads();
        }
        // epilogue of the owned nodes of plane zz
        const long long plane = (long long)zz * NY;
        for (int idx = tid; idx < kOwnX * kOwnY * kLG; idx += kTcThreads) {
            const int r = 1 + idx / (kOwnX * kLG), rem = idx % (kOwnX * kLG);
            const int cx = 1 + rem / kLG, le = rem % kLG;
            const int gxn = x0e + cx, gyn = y0e + r;
            if (gxn >= NX || gyn >= NY) continue;
            const long long n = (plane + gyn) * a.px + gxn;
            const long long rec = GMG_B(n * kLoads + kLG * lg + le, (long long)a.px * NY * NZ * kLoads, 551);
            const float4 yv = NF[(r * kTNX + cx) * kLG + le];
            const uint8_t m = a.maskp[n];
            const bool f0 = !fbit(m, 0), f1 = !fbit(m, 1), f2 = !fbit(m, 2);
            float4* out = reinterpret_cast<float4*>(a.out) + rec;
            if (MODE == FM_APPLY) {
                const float4 v = make_float4(f0 ? yv.x : 0.f, f1 ? yv.y : 0.f, f2 ? yv.z : 0.f, 0.f);
                *out = v;
                if (DOT) {
                    const float4 xv = reinterpret_cast<const float4*>(a.xin)[rec];
                    dotv.add_prod(f0 ? xv.x : 0.f, v.x);
                    dotv.add_prod(f1 ? xv.y : 0.f, v.y);
                    dotv.add_prod(f2 ? xv.z : 0.f, v.z);
                }
            } else if (MODE == FM_RESID) {
                const float4 bv = reinterpret_cast<const float4*>(a.b)[rec];
                *out = make_float4(f0 ? bv.x - yv.x : 0.f, f1 ? bv.y - yv.y : 0.f, f2 ? bv.z - yv.z : 0.f, 0.f);
            } else {
                const float4 bv = reinterpret_cast<const float4*>(a.b)[rec];
                const float4 xv = reinterpret_cast<const float4*>(a.xin)[rec];
                const float inv = a.inv0[n];
                float d0 = ca * inv * (bv.x - yv.x), d1 = ca * inv * (bv.y - yv.y), d2 = ca * inv * (bv.z - yv.z);
                if (cd != 0.f) {
                    const float4 dv = reinterpret_cast<const float4*>(a.dold)[rec];
                    d0 = fmaf(cd, dv.x, d0);
                    d1 = fmaf(cd, dv.y, d1);
                    d2 = fmaf(cd, dv.z, d2);
                }
                d0 = f0 ? d0 : 0.f;
                d1 = f1 ? d1 : 0.f;
                d2 = f2 ? d2 : 0.f;
                const float4 xn = make_float4(f0 ? xv.x + d0 : 0.f, f1 ? xv.y + d1 : 0.f, f2 ? xv.z + d2 : 0.f, 0.f);
                *out = xn;
                if (a.dnew) reinterpret_cast<float4*>(a.dnew)[rec] = make_float4(d0, d1, d2, 0.f);
                if (DOT) {
                    dotv.add_prod(f0 ? bv.x : 0.f, xn.x);
                    dotv.add_prod(f1 ? bv.y : 0.f, xn.y);
                    dotv.add_prod(f2 ? bv.z : 0.f, xn.z);
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < kPlaneRec; i += kTcThreads) NF[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    };

    // ---- prologue: planes kb .. kb + 2, split of plane kb
    if (tid == 0) {
        issue_plane(kb);
        issue_plane(kb + 1);
        issue_plane(kb + 2);
    }
    bool failed = !wait_plane(kb);
    split(kb);
    // ---- layers kb .. k1 - 1: MMAs of layer z, forces of layer z - 1
    for (int z = kb; z < k1; ++z) {
        if (!wait_plane(z + 1)) failed = true;
        split(z + 1);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        if (tid == 0) issue_mma(z);
        if (z > kb) {
            if (!wait_mma(z - 1)) failed = true;
            if (tid == 0 && z + 2 <= k1) issue_plane(z + 2);  // the slot of plane z - 1, read by MMA z - 1 only
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            process(z - 1);
        }
    }
    if (!failed) {
        if (!wait_mma(k1 - 1)) failed = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        process(k1 - 1);
    }
    if (__syncthreads_or(failed)) {
        // drain: every copy and MMA commit issued must complete before the
        // shared memory and TMEM are released
        if (tid == 0) {
            for (int p = p_con + 1; p <= p_iss; ++p) wait_bar(&tbar[slot_of(p)], (unsigned)(((p - kb) / 3) & 1));
            for (int z = z_con + 1; z <= z_iss; ++z) wait_bar(&mbar[(z - kb) & 1], (unsigned)(((z - kb) >> 1) & 1));
            atomicExch(a.err, 1);
        }
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
        return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    if (DOT) {
        // per load: lanes with the same tid % 8, then the 16 warps in order
        double v = dotv.value();
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (lane < kLG) red[warp * kLG + lane] = v;
        __syncthreads();
        if (tid < kLG) {
            double s = 0.0;
            for (int w = 0; w < 16; ++w) s += red[w * kLG + tid];
            a.partial[(long long)(kLG * lg + tid) * a.pstride + tile] = s;
        }
    }
}

struct TcPlan {
    int gx, gy, gz, zc;
};

int tc_sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

// Tiles of 15 x 7 owned nodes; the z-chunk that minimises (waves x layers per
// CTA) with one CTA per SM and both load groups.
TcPlan tc_plan(int nx, int ny, int nz, int ngroups) {
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int gx = (NX + kOwnX - 1) / kOwnX, gy = (NY + kOwnY - 1) / kOwnY;
    const int slots = tc_sm_count();
    TcPlan best{gx, gy, 1, NZ};
    long long best_cost = -1;
    for (int nch = 1; nch <= NZ; ++nch) {
        const int zc = (NZ + nch - 1) / nch;
        if (zc < 4 && nch > 1) break;
        const int gz = (NZ + zc - 1) / zc;
        const long long blocks = (long long)gx * gy * gz * ngroups;
        const long long cost = ((blocks + slots - 1) / slots) * (zc + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = TcPlan{gx, gy, gz, zc};
        }
    }
    return best;
}

template <int MODE, bool DOT, int PASSES>
int tc_launch(const TcPlan& pl, int ngroups, const MFineArgs& a, const float* Bop, float scale, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_mfine_tc<MODE, DOT, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) !=
            cudaSuccess)
            return GMG_ERR_CUDA;
        attr = true;
    }
    const int NX = a.nx + 1, NY = a.ny + 1, NZ = a.nz + 1;
    const unsigned long long vd[4] = {(unsigned long long)kNodeF, (unsigned long long)NX, (unsigned long long)NY,
                                      (unsigned long long)NZ};
    const unsigned long long vs[3] = {4ull * kNodeF, 4ull * kNodeF * a.px, 4ull * kNodeF * a.px * NY};
    const unsigned bx[4] = {(unsigned)(4 * kLG), (unsigned)kTNX, (unsigned)kTNY, 1u};
    const unsigned long long ed[3] = {(unsigned long long)a.nx, (unsigned long long)a.ny, (unsigned long long)a.nz};
    const unsigned long long es[2] = {4ull * a.epitch, 4ull * a.epitch * a.ny};
    const unsigned be[3] = {(unsigned)kEW, (unsigned)kTEY, 1u};
    CUtensorMap mx, me;
    if (!encode_f32_map_strided(&mx, a.xin, 4, vd, vs, bx) || !encode_f32_map_strided(&me, a.Ep, 3, ed, es, be))
        return GMG_ERR_CUDA;
    note_launch();
    pdl_launch(k_mfine_tc<MODE, DOT, PASSES>, dim3((unsigned)(pl.gx * pl.gy * pl.gz * ngroups)), dim3(kTcThreads),
               (size_t)kSmem, s, mx, me, a, Bop, scale, pl.zc, pl.gx, pl.gy, ngroups);
    return GMG_OK;
}

template <int MODE, bool DOT>
int tc_launch_p(const TcPlan& pl, int ngroups, const MFineArgs& a, const float* Bop, float scale, int passes,
                cudaStream_t s) {
    return passes > 3 ? tc_launch<MODE, DOT, 5>(pl, ngroups, a, Bop, scale, s)
                      : tc_launch<MODE, DOT, 3>(pl, ngroups, a, Bop, scale, s);
}

// standard local index of the corner at offset (dx, dy, dz)
int corner_std(int dx, int dy, int dz) { return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0)); }

float host_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

}  // namespace

int mfine_tc_blocks(int nx, int ny, int nz) {
    const TcPlan pl = tc_plan(nx, ny, nz, 2);
    return pl.gx * pl.gy * pl.gz;
}

int launch_mfine_tc(int mode, int dot, const MFineArgs& a, const float* Bop, float scale, int passes,
                    cudaStream_t s) {
    const int ngroups = a.nl > kLG ? 2 : 1;
    const TcPlan pl = tc_plan(a.nx, a.ny, a.nz, 2);  // the same tiles for any load count (partial layout)
    if (mode == FM_APPLY)
        return dot ? tc_launch_p<FM_APPLY, true>(pl, ngroups, a, Bop, scale, passes, s)
                   : tc_launch_p<FM_APPLY, false>(pl, ngroups, a, Bop, scale, passes, s);
    if (mode == FM_SMOOTH)
        return dot ? tc_launch_p<FM_SMOOTH, true>(pl, ngroups, a, Bop, scale, passes, s)
                   : tc_launch_p<FM_SMOOTH, false>(pl, ngroups, a, Bop, scale, passes, s);
    return tc_launch_p<FM_RESID, false>(pl, ngroups, a, Bop, scale, passes, s);
}

int build_mfine_tc_operand(const double* Ke, float* out, float* scale_out) {
    // K_e = s * Kint with |Kint| < 2048 integers (exact in TF32), if it is one
    double s = 1.0;
    bool exact = false;
    for (int k0 = 1; k0 < 2048 && !exact; ++k0) {
        s = Ke[0] / k0;
        exact = true;
        for (int i = 0; i < 576 && exact; ++i) {
            const double v = Ke[i] / s, r = std::nearbyint(v);
            exact = std::fabs(v - r) <= 1e-9 * std::max(1.0, std::fabs(r)) && std::fabs(r) < 2048.0;
        }
    }
    if (!exact) s = 1.0;
    std::memset(out, 0, sizeof(float) * 2048);
    for (int j = 0; j < 4; ++j) {
        const int dy = j & 1, dz = j >> 1;
        for (int dx = 0; dx < 2; ++dx)
            for (int o = 0; o < 24; ++o) {
                const int ao = o / 3, co = o % 3;
                const int row = 3 * corner_std(ao & 1, (ao >> 1) & 1, ao >> 2) + co;
                for (int c = 0; c < 3; ++c) {
                    const int col = 3 * corner_std(dx, dy, dz) + c;
                    const double v = Ke[row * 24 + col] / s;
                    const int idx = j * 256 + dx * 128 + o * 4 + c;
                    if (exact) {
                        out[idx] = (float)std::nearbyint(v);
                    } else {
                        const float hi = host_tf32((float)v);
                        out[idx] = hi;
                        out[1024 + idx] = (float)(v - (double)hi);
                    }
                }
            }
    }
    *scale_out = (float)s;
    return exact ? 3 : 5;
}

}  // namespace gmg
