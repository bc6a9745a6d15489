// Level 1 of the hierarchy applied matrix-free (the Galerkin operator of
// Eq. galerkin_level1 evaluated per coarse element instead of read from its
// assembled planes), for sm_103a.
//
// Formulation.  For even fine sizes every coarse element is the union of 8 fine
// children, child k = (kx, ky, kz) in {0, 1}^3, and
//     K^1_c = sum_k E_k P_k^T K_e P_k,
// with P_k the trilinear prolongation from the coarse element's 8 corners to
// child k's 8 nodes.  In the Walsh-Hadamard mode basis of the coarse corners
// (modes (m, c): monomial m of the corner signs, component c, as in fine.cu),
// child k is the reflection of child 0 through the axes set in k, and a
// reflection only flips the signs of the modes whose parity has those axes:
//     H P_k^T K_e P_k H^T / 64 = D_k G0 D_k,   D_k = diag((-1)^{k . pi(m, c)}),
// where pi(m, c) is the parity of mode (m, c) under the three reflections and
//     G0 = T0^T G T0
// (G the fine element's parity blocks, T0 the prolongation to child 0 in the
// mode basis: child monomial a takes coarse monomials m that contain a, with
// weight prod over axes of 1 (a_x = m_x = 0), -1/2 (a_x = 0, m_x = 1) or 1/2
// (a_x = m_x = 1)).  Summing over the children,
//     (K^1_c)_{ij} = G0_{ij} * Ehat[pi_i xor pi_j],
//     Ehat[d] = sum_k E_k (-1)^{popcount(k & d)}    (8-point Hadamard transform
//                                                    of the children's moduli).
// G0 has 279 non-zero entries for every Poisson ratio (none in the constant
// modes): the pattern is fixed by the structure of G and T0 and is built at
// compile time below; the 279 values are computed on the host from the FP64
// blocks of G.  One coarse element costs the 21 mode sums, 279 multiply-adds
// grouped by parity difference, about 160 products with Ehat, and the
// transform back to corners; the assembled kernel reads 126 x 4 bytes of
// operator per node instead.
//
// Exactness.  The sum equals the assembled level-1 operator on the free DOFs
// when every fixed fine DOF has only fixed coarse DOFs among its prolongation
// parents (then the masked prolongation acts on vectors that vanish on fixed
// coarse DOFs as the unmasked one does); the host checks this and the even
// sizes before choosing the kernel, and the assembled kernel serves every
// other grid.
//
// Schedule.  Level 1 has an eighth of the fine elements, too few for the fine
// kernel's column-per-thread z-march to fill the GPU without recomputing tile
// halos and chunk boundaries (that form computed 2.2 elements per element and
// took 20 us at 100^3).  Two launches instead:
//   - k_l1mf_elem, one thread per coarse element in linear order: the block's
//     corner nodes (two contiguous index ranges) are staged in shared memory
//     with fixed DOFs zeroed; each thread transforms its 8 corners to modes
//     (a 3-stage Walsh-Hadamard butterfly per component), applies the
//     Ehat-weighted G0 (coefficients as kernel parameters), transforms back
//     and writes its 8 corner forces as float4 records, corner-major;
//   - k_l1mf_node, one thread per node: the corner forces of its up to 8 cells
//     added in a fixed order (the 16 MB of records stay in L2), then the
//     level's epilogue (apply, residual or smoother step).
// Every add, subtract and product is rounded on its own.
#include <algorithm>
#include <cmath>
#include <utility>

#include "internal.cuh"

namespace gmg {

namespace {

// ---- the compile-time pattern of G0 ------------------------------------------
// Monomial (bit 0 = X, 1 = Y, 2 = Z) of component c in parity class sigma (as fine.cu).
constexpr int l1_mono(int sigma, int c) {
    return ((sigma & 1) ^ (c == 0 ? 1 : 0)) | ((((sigma >> 1) & 1) ^ (c == 1 ? 1 : 0)) << 1) |
           ((((sigma >> 2) & 1) ^ (c == 2 ? 1 : 0)) << 2);
}
// Parity of mode (m, c) under the reflections x, y, z (bit a flips when the
// monomial contains axis a, and once more for the component along a).
constexpr int l1_parity(int m, int c) { return m ^ (1 << c); }

// Whether entry (row r, column s) of G's parity block sigma is non-zero for a
// generic Poisson ratio (the symmetric form of G: classes 0 and 7 full; 1, 2
// and 4 the 2x2 block of their two non-constant components; 3, 5 and 6 the
// 2x2 block of equal entries and the XYZ diagonal).
constexpr bool l1_gsym_nonzero(int sigma, int r, int s) {
    if (sigma == 0 || sigma == 7) return true;
    if (sigma == 1 || sigma == 2 || sigma == 4) {
        const int skip = sigma == 1 ? 0 : (sigma == 2 ? 1 : 2);  // the component with the constant monomial
        return r != skip && s != skip;
    }
    const int dr = sigma == 3 ? 2 : (sigma == 5 ? 1 : 0);        // the XYZ row
    return (r == dr) == (s == dr);
}
// G's structural non-zero between modes (a, c) and (b, c2): the parity of a
// mode is its class (l1_mono(parity, c) == a).
constexpr bool l1_g_nonzero(int a, int c, int b, int c2) {
    if (l1_parity(a, c) != l1_parity(b, c2)) return false;
    return l1_gsym_nonzero(l1_parity(a, c), c, c2);
}

constexpr int kL1Modes = 24;  // (m, c) -> 3 m + c

// Which of the eight values of G's symmetric form (0 a, 1 b of class 0; 2 a',
// 3 b' of class 7; 4 p, 5 q of classes 1, 2, 4; 6 c, 7 d of classes 3, 5, 6)
// G couples modes (a, c) and (b, c2) with, or -1.
constexpr int l1_g_value(int a, int c, int b, int c2) {
    if (!l1_g_nonzero(a, c, b, c2)) return -1;
    const int sigma = l1_parity(a, c);
    if (sigma == 0) return c == c2 ? 0 : 1;
    if (sigma == 7) return c == c2 ? 2 : 3;
    if (sigma == 1 || sigma == 2 || sigma == 4) return c == c2 ? 4 : 5;
    const int dr = sigma == 3 ? 2 : (sigma == 5 ? 1 : 0);
    return c == dr ? 7 : 6;
}
// T0: child monomial a from coarse monomial m (per axis 1, -1/2 or 1/2; 0 when
// a is not inside m).  Products of these are exact in double.
constexpr double l1_t0(int a, int m) {
    double w = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        const int ab = (a >> ax) & 1, mb = (m >> ax) & 1;
        if (ab && !mb) return 0.0;
        if (mb) w *= ab ? 0.5 : -0.5;
    }
    return w;
}

struct L1Pattern {
    int count, classes;
    int i[kL1Coefs], j[kL1Coefs], d[kL1Coefs];
    int cls[kL1Coefs];   // the entry equals (neg ? -1 : 1) * class value cls
    bool neg[kL1Coefs];
    double w[kL1Coefs][8];  // the entry as a combination of G's eight values
};
// Entries (i, j) of G0 = T0^T G T0 with some a inside m_i and b inside m_j
// coupled by G, sorted by row, then parity difference, then column; each entry
// is the combination sum_{a, b} T0[a][m_i] G_ab T0[b][m_j] of G's eight values,
// and entries with the same combination up to sign share a class (equal for
// every Poisson ratio).
constexpr L1Pattern l1_make_pattern() {
    L1Pattern p{};
    p.count = 0;
    p.classes = 0;
    int rep[kL1Coefs] = {};  // the first entry of each class
    for (int i = 0; i < kL1Modes; ++i)
        for (int d = 0; d < 8; ++d)
            for (int j = 0; j < kL1Modes; ++j) {
                const int mi = i / 3, ci = i % 3, mj = j / 3, cj = j % 3;
                if ((l1_parity(mi, ci) ^ l1_parity(mj, cj)) != d) continue;
                double w[8] = {};
                bool nz = false;
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) {
                        const int g = l1_g_value(a, ci, b, cj);
                        if ((a & ~mi) == 0 && (b & ~mj) == 0 && g >= 0) {
                            w[g] += l1_t0(a, mi) * l1_t0(b, mj);
                            nz = true;
                        }
                    }
                if (!nz) continue;
                if (p.count < kL1Coefs) {
                    const int n = p.count;
                    p.i[n] = i;
                    p.j[n] = j;
                    p.d[n] = d;
                    for (int k = 0; k < 8; ++k) p.w[n][k] = w[k];
                    int c = -1;
                    bool ng = false;
                    for (int q = 0; q < p.classes && c < 0; ++q) {
                        bool same = true, opp = true;
                        for (int k = 0; k < 8; ++k) {
                            same = same && p.w[rep[q]][k] == w[k];
                            opp = opp && p.w[rep[q]][k] == -w[k];
                        }
                        if (same || opp) {
                            c = q;
                            ng = !same;
                        }
                    }
                    if (c < 0) {
                        c = p.classes++;
                        rep[c] = n;
                    }
                    p.cls[n] = c;
                    p.neg[n] = ng;
                }
                ++p.count;
            }
    return p;
}
constexpr L1Pattern kL1Pat = l1_make_pattern();
static_assert(kL1Pat.count == kL1Coefs, "G0 has 279 structural non-zeros");
static_assert(kL1Pat.classes == kL1Classes, "G0's entries take 21 values up to sign");

}  // namespace

namespace {

// ---- the element contraction -----------------------------------------------------
// w_i = sum over the pattern of Ehat[d] * (sum_j G0_ij v_j), one group per
// (row, parity difference): the group's products and sums are rounded in the
// pattern's order, then scaled by Ehat[d] and added to the row.
struct L1Acc {
    float t, acc;
};
// first entry of the (row, parity difference) group of entry n
__host__ __device__ constexpr int l1_group_start(int n) {
    while (n > 0 && kL1Pat.i[n - 1] == kL1Pat.i[n] && kL1Pat.d[n - 1] == kL1Pat.d[n]) --n;
    return n;
}
template <int N>
__device__ __forceinline__ void l1_term(L1Acc& s, const float (&G)[kL1Classes], const float (&v)[kL1Modes],
                                        const float (&eh)[8], float (&w)[kL1Modes]) {
    constexpr int I = kL1Pat.i[N], J = kL1Pat.j[N], D = kL1Pat.d[N], C = kL1Pat.cls[N];
    constexpr bool NEG = kL1Pat.neg[N];
    constexpr int S = l1_group_start(N);
    constexpr bool grp_first = S == N;
    constexpr bool row_first_group = S == 0 || kL1Pat.i[S - 1] != I;  // the row's first group
    constexpr bool row_last = N + 1 == kL1Coefs || kL1Pat.i[N + 1] != I;
    constexpr bool grp_last = row_last || kL1Pat.d[N + 1] != D;
    const float g = NEG ? -G[C] : G[C];
    s.t = grp_first ? __fmul_rn(g, v[J]) : __fmaf_rn(g, v[J], s.t);
    if (grp_last) s.acc = row_first_group ? __fmul_rn(eh[D], s.t) : __fmaf_rn(eh[D], s.t, s.acc);
    if (row_last) w[I] = s.acc;
}
template <int... Ns>
__device__ __forceinline__ void l1_terms(std::integer_sequence<int, Ns...>, const float (&G)[kL1Classes],
                                         const float (&v)[kL1Modes], const float (&eh)[8], float (&w)[kL1Modes]) {
    L1Acc s{0.f, 0.f};
    (l1_term<Ns>(s, G, v, eh, w), ...);
}

}  // namespace

namespace {

constexpr int kL1Threads = 128;

template <int NTH>
__device__ __forceinline__ double l1_block_sum(double v, int tid) {
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

// 8-point Walsh-Hadamard transform over the corner bits (x = bit 0): forward
// (corners q -> modes m, v_m = sum_q prod_{k in m} s_k(q) u_q, s_k = -1 on the
// low side) and its transpose (modes -> corner forces).
__device__ __forceinline__ void l1_wht(float (&u)[8]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (!(q & (1 << k))) {
                const float a = u[q], b = u[q | (1 << k)];
                u[q] = __fadd_rn(a, b);
                u[q | (1 << k)] = __fsub_rn(b, a);
            }
}
__device__ __forceinline__ void l1_wht_t(float (&w)[8]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (!(q & (1 << k))) {
                const float c = w[q], l = w[q | (1 << k)];
                w[q] = __fsub_rn(c, l);
                w[q | (1 << k)] = __fadd_rn(c, l);
            }
}

// Phase 1, one thread per coarse element, elements in their linear order.
// The block's corner nodes lie in two contiguous index ranges (the low plane
// of its elements and the same range one node plane up); they are staged in
// shared memory with fixed DOFs zeroed.  Each thread takes its 8 corner values
// to modes, applies the Ehat-weighted G0 and writes the 8 corner forces back as
// float4 records cf[q][e] (q = qx + 2 qy + 4 qz; w unused).
// Nodes per staged range of any block of kL1Threads consecutive elements: the
// low corners advance by 1 per element, 2 at a row end and nx + 3 at a plane
// end, plus the row and node of the high corners.
__host__ __device__ inline long long l1_span_bound(int nx, int ny) {
    return kL1Threads - 1 + (kL1Threads - 1) / nx + 1 + ((kL1Threads - 1) / ((long long)nx * ny) + 1) * (nx + 2) +
           nx + 1 + 2;
}
__global__ void __launch_bounds__(kL1Threads) k_l1mf_elem(BsrArgs a, const __grid_constant__ L1Coef G, float4* cf,
                                                           int stage) {
    extern __shared__ float4 sn[];  // [stage]: 2 ranges of at most stage / 2 nodes
    pdl_entry();
    // 32-bit indices throughout (set-up admits level 1 only with 8 ne < 2^31)
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int ne = nx * ny * nz, nxy = nx * ny;
    const int NX = nx + 1, NXY = NX * (ny + 1), nn = (int)a.nn;
    const int e_first = blockIdx.x * kL1Threads;
    const int e_last = (e_first + kL1Threads < ne ? e_first + kL1Threads : ne) - 1;
    auto low_node = [&](int e) {
        const int k = e / nxy, r = e - k * nxy, j = r / nx;
        return (r - j * nx) + NX * j + NXY * k;
    };
    const int lo = low_node(e_first);
    const int span = low_node(e_last) + NX + 2 - lo;  // nodes per range
    for (int t = threadIdx.x; t < 2 * span; t += kL1Threads) {
        const int n = lo + (t < span ? t : t - span + NXY);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < nn) {
            const int m = __ldg(a.mask + n);
            const float x = __ldg(a.xin + 3 * n), y = __ldg(a.xin + 3 * n + 1), z = __ldg(a.xin + 3 * n + 2);
            v = make_float4((m & 1) ? 0.f : x, (m & 2) ? 0.f : y, (m & 4) ? 0.f : z, 0.f);
        }
        sn[GMG_B(t, stage, 617)] = v;
    }
    __syncthreads();
    const int e = e_first + threadIdx.x;
    if (e >= ne) return;
    const int r0 = low_node(e) - lo;
    float u[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int r = r0 + (q & 1) + NX * ((q >> 1) & 1) + ((q >> 2) & 1) * span;
        const float4 v = sn[GMG_B(r, stage, 618)];
        u[0][q] = v.x;
        u[1][q] = v.y;
        u[2][q] = v.z;
    }
    float eh[8];
    {
        const float4* p = reinterpret_cast<const float4*>(a.eh) + GMG_B(2 * e, 2LL * ne, 613);
        const float4 e0 = __ldg(p), e1 = __ldg(p + 1);
        eh[0] = e0.x; eh[1] = e0.y; eh[2] = e0.z; eh[3] = e0.w;
        eh[4] = e1.x; eh[5] = e1.y; eh[6] = e1.z; eh[7] = e1.w;
    }
    float v[kL1Modes], w[kL1Modes];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        l1_wht(u[c]);
#pragma unroll
        for (int m = 0; m < 8; ++m) v[3 * m + c] = u[c][m];
    }
#pragma unroll
    for (int i = 0; i < kL1Modes; ++i) w[i] = 0.f;
    float gc[kL1Classes];  // the 21 class values, in registers for the whole contraction
#pragma unroll
    for (int k = 0; k < kL1Classes; ++k) gc[k] = G.g[k];
    l1_terms(std::make_integer_sequence<int, kL1Coefs>{}, gc, v, eh, w);
    float f[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int m = 0; m < 8; ++m) f[c][m] = w[3 * m + c];
        l1_wht_t(f[c]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) cf[GMG_B(q * ne + e, 8LL * ne, 615)] = make_float4(f[0][q], f[1][q], f[2][q], 0.f);
}

// Phase 2, one thread per node: the corner forces of its (up to 8) cells added
// in a fixed order, then the epilogue (apply / residual / smoother step, with
// the optional dot product).
template <int MODE, bool DOT>
__global__ void __launch_bounds__(kL1Threads) k_l1mf_node(BsrArgs a, const float4* cf) {
    pdl_entry();
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nn = (int)a.nn, ne = nx * ny * nz;
    const int n = blockIdx.x * kL1Threads + threadIdx.x;
    DSAcc dotv;
    if (n < nn) {
        const int NX = nx + 1, NXY = NX * (ny + 1);
        const int k = n / NXY, r = n - k * NXY, j = r / NX, i = r - j * NX;
        float y[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // this node is corner q of element (i - qx, j - qy, k - qz)
            const int I = i - (q & 1), J = j - ((q >> 1) & 1), K = k - ((q >> 2) & 1);
            const bool ok = I >= 0 && I < nx && J >= 0 && J < ny && K >= 0 && K < nz;
            const int e = ok ? I + nx * (J + ny * K) : 0;
            const float4 f = __ldg(cf + GMG_B(q * ne + e, 8LL * ne, 616));
            y[0] = __fadd_rn(y[0], ok ? f.x : 0.f);
            y[1] = __fadd_rn(y[1], ok ? f.y : 0.f);
            y[2] = __fadd_rn(y[2], ok ? f.z : 0.f);
        }
        const int msk = a.mask[n];
        if (MODE == FM_APPLY) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fr = !((msk >> c) & 1);
                const float v = fr ? y[c] : 0.f;
                a.out[3 * n + c] = v;
                if (DOT) dotv.add_prod(fr ? a.xin[3 * n + c] : 0.f, v);
            }
        } else if (MODE == FM_RESID) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                a.out[3 * n + c] = ((msk >> c) & 1) ? 0.f : __fsub_rn(a.b[3 * n + c], y[c]);
        } else {
            const float cd = (float)a.coef[2 * a.step], ca = (float)a.coef[2 * a.step + 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float xn = 0.f, dn = 0.f;
                if (!((msk >> c) & 1)) {
                    const float bc = a.b[3 * n + c];
                    dn = __fmul_rn(__fmul_rn(ca, a.invdiag[3 * n + c]), __fsub_rn(bc, y[c]));
                    if (cd != 0.f) dn = fmaf(cd, a.dold[3 * n + c], dn);
                    xn = __fadd_rn(a.xin[3 * n + c], dn);
                    if (DOT) dotv.add_prod(bc, xn);
                }
                a.out[3 * n + c] = xn;
                if (a.dnew) a.dnew[3 * n + c] = dn;
            }
        }
    }
    if (DOT) {
        const double sum = l1_block_sum<kL1Threads>(dotv.value(), threadIdx.x);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = sum;
    }
}

}  // namespace

namespace {

// Ehat of every coarse element from its 8 children's FP64 moduli (the fine
// level has even sizes): Ehat[d] = sum_k E_k (-1)^{popcount(k & d)}, child k =
// (kx, ky, kz) at fine element (2I + kx, 2J + ky, 2K + kz).
__global__ void k_l1_ehat(const double* E, int nx, int ny, int nz, float* eh) {
    const int cnx = nx / 2, cny = ny / 2, cnz = nz / 2;
    const long long ne = (long long)cnx * cny * cnz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(e % cnx), J = (int)((e / cnx) % cny), K = (int)(e / ((long long)cnx * cny));
        double Ek[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long f = (2 * I + (k & 1)) + (long long)nx * ((2 * J + ((k >> 1) & 1)) +
                                                                     (long long)ny * (2 * K + ((k >> 2) & 1)));
            Ek[k] = E[f];
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) s += (__popc(k & d) & 1) ? -Ek[k] : Ek[k];
            eh[8 * e + d] = (float)s;
        }
    }
}

}  // namespace

int l1mf_grid_blocks(int nx, int ny, int nz) {
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    return (int)((nn + kL1Threads - 1) / kL1Threads);
}

void launch_l1mf(int mode, int dot, const BsrArgs& a, const L1Coef& G, float* cf_buf, cudaStream_t s) {
    float4* cf = reinterpret_cast<float4*>(cf_buf);
    const long long ne = (long long)a.nx * a.ny * a.nz;
    const dim3 ge((unsigned)((ne + kL1Threads - 1) / kL1Threads)), gn((unsigned)l1mf_grid_blocks(a.nx, a.ny, a.nz));
    const int stage = (int)(2 * l1_span_bound(a.nx, a.ny));
    note_launch(2);
    pdl_launch(k_l1mf_elem, ge, dim3(kL1Threads), sizeof(float4) * (size_t)stage, s, a, G, cf, stage);
    if (mode == FM_APPLY) {
        if (dot) pdl_launch(k_l1mf_node<FM_APPLY, true>, gn, dim3(kL1Threads), 0, s, a, (const float4*)cf);
        else pdl_launch(k_l1mf_node<FM_APPLY, false>, gn, dim3(kL1Threads), 0, s, a, (const float4*)cf);
    } else if (mode == FM_SMOOTH) {
        if (dot) pdl_launch(k_l1mf_node<FM_SMOOTH, true>, gn, dim3(kL1Threads), 0, s, a, (const float4*)cf);
        else pdl_launch(k_l1mf_node<FM_SMOOTH, false>, gn, dim3(kL1Threads), 0, s, a, (const float4*)cf);
    } else {
        pdl_launch(k_l1mf_node<FM_RESID, false>, gn, dim3(kL1Threads), 0, s, a, (const float4*)cf);
    }
}

void launch_l1_ehat(const double* E_fine, int nx, int ny, int nz, float* eh, cudaStream_t s) {
    note_launch();
    k_l1_ehat<<<148 * 4, 256, 0, s>>>(E_fine, nx, ny, nz, eh);
}

bool l1_coef_from_blocks(const double g[72], L1Coef* out) {
    // G in the mode basis (3 m + c): block entry (sigma, r, s) couples modes
    // (mono(sigma, r), r) and (mono(sigma, s), s)
    double Gm[kL1Modes][kL1Modes] = {};
    for (int sig = 0; sig < 8; ++sig)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const int mr = l1_mono(sig, r), mc = l1_mono(sig, c);
                if (mr == 0 || mc == 0) continue;
                Gm[3 * mr + r][3 * mc + c] = g[sig * 9 + r * 3 + c];
            }
    // T0: child monomial a from coarse monomial m (a inside m), same component
    auto t0 = [](int a, int m) {
        double w = 1.0;
        for (int ax = 0; ax < 3; ++ax) {
            const int ab = (a >> ax) & 1, mb = (m >> ax) & 1;
            if (ab && !mb) return 0.0;
            if (mb) w *= ab ? 0.5 : -0.5;
        }
        return w;
    };
    double G0[kL1Modes][kL1Modes] = {};
    double big = 0.0;
    for (int i = 0; i < kL1Modes; ++i)
        for (int j = 0; j < kL1Modes; ++j) {
            double s = 0.0;
            for (int a = 0; a < 8; ++a) {
                const double ta = t0(a, i / 3);
                if (ta == 0.0) continue;
                for (int b = 0; b < 8; ++b) {
                    const double tb = t0(b, j / 3);
                    if (tb != 0.0) s += ta * Gm[3 * a + i % 3][3 * b + j % 3] * tb;
                }
            }
            G0[i][j] = s;
            big = std::max(big, std::fabs(s));
        }
    bool inpat[kL1Modes][kL1Modes] = {};
    double cv[kL1Classes] = {};
    bool have[kL1Classes] = {};
    for (int n = 0; n < kL1Coefs; ++n) {
        const double v = G0[kL1Pat.i[n]][kL1Pat.j[n]] * (kL1Pat.neg[n] ? -1.0 : 1.0);
        inpat[kL1Pat.i[n]][kL1Pat.j[n]] = true;
        if (!have[kL1Pat.cls[n]]) {
            cv[kL1Pat.cls[n]] = v;
            have[kL1Pat.cls[n]] = true;
        } else if (std::fabs(v - cv[kL1Pat.cls[n]]) > 1e-12 * big) {
            return false;  // a class whose entries differ: G lacks the assumed structure
        }
    }
    for (int k = 0; k < kL1Classes; ++k) out->g[k] = (float)cv[k];
    for (int i = 0; i < kL1Modes; ++i)
        for (int j = 0; j < kL1Modes; ++j)
            if (!inpat[i][j] && std::fabs(G0[i][j]) > 1e-12 * big) return false;
    return big > 0.0;
}

bool l1mf_eligible(int nx, int ny, int nz, const uint8_t* fine_mask_host) {
    if (nx % 2 || ny % 2 || nz % 2 || nx < 2 || ny < 2 || nz < 2) return false;
    if (8LL * (nx / 2) * (ny / 2) * (nz / 2) >= (1LL << 31) - 1) return false;  // the kernels' 32-bit indices
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    // every fixed fine DOF: all of its prolongation parents' DOFs fixed (the
    // parents' fixed bits are the fine bits at their injection nodes)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                const int m = fine_mask_host[i + (long long)NX * (j + (long long)NY * k)];
                if (m == 0) continue;
                const int i0 = i & ~1, i1 = (i & 1) ? i + 1 : i, j0 = j & ~1, j1 = (j & 1) ? j + 1 : j;
                const int k0 = k & ~1, k1 = (k & 1) ? k + 1 : k;
                for (int pk = k0; pk <= k1; pk += 2)
                    for (int pj = j0; pj <= j1; pj += 2)
                        for (int pi = i0; pi <= i1; pi += 2) {
                            const int pm = fine_mask_host[pi + (long long)NX * (pj + (long long)NY * pk)];
                            if ((pm & m) != m) return false;
                        }
            }
    return true;
}

}  // namespace gmg
