// Learned warm start: a 3-D convolutional encoder-decoder trained and run by
// this library's own kernels (include/gmg_warmnet.h states the network, the
// layouts and the arithmetic).
//
// Kernels (all channels-last, FP32 activations and accumulation, weights held
// as bfloat16-rounded values in FP32 containers):
//   k_conv<COB,TY,TZ,S>  direct 3x3x3 convolution, stride 1 or 2: a block owns
//                        an 8 x TY x TZ tile of output nodes and COB output
//                        channels; per chunk of 4 input channels it stages the
//                        input halo (planar, odd x pitch) and the weights in
//                        shared memory; each thread keeps 8 consecutive x
//                        outputs x 4 channels in registers and loads each halo
//                        row once for its three x taps.  Also serves the
//                        backward data pass of stride-1 layers (weights
//                        transposed and flipped) with an accumulate flag and a
//                        leaky-ReLU-derivative epilogue;
//   k_conv_s2t<CIG>      backward data pass of a stride-2 layer (transposed
//                        convolution: each fine node gathers from 1, 2, 4 or 8
//                        taps by the parity of its coordinates);
//   k_wgrad<S>           weight and bias gradients: one thread per (4 output
//                        channels, 4 input channels, tap), a split of the
//                        batch's output nodes per block, partial sums written
//                        per split and added in a fixed order by k_sum_splits;
//   k_upsample / k_upsample_adj   trilinear prolongation into a concatenation
//                        slice and its adjoint (times the activation derivative);
//   loss, Adam, features, target and warm-start kernels.
// Every reduction has a fixed order, so a step is bitwise reproducible.

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gmg_warmnet.h"
#include "internal.cuh"

namespace {

using gmg::note_launch;
using gmg::smem_u32;
using gmg::mbar_init;
using gmg::mbar_fence_init;
using gmg::mbar_expect_tx;
using gmg::mbar_try_wait;

constexpr float kSlope = 0.1f;
constexpr double kBeta1 = 0.9, kBeta2 = 0.999, kAdamEps = 1e-8;
constexpr int kLayers = GMG_NET_LAYERS;

struct LayerDef {
    int cin, cout, stride, act;
};
constexpr LayerDef kDefs[kLayers] = {{12, 16, 1, 1},  {16, 16, 1, 1}, {16, 32, 2, 1},  {32, 32, 1, 1},
                                     {32, 64, 2, 1}, {64, 64, 1, 1}, {64, 64, 2, 1},  {64, 64, 1, 1},
                                     {128, 64, 1, 1}, {96, 32, 1, 1}, {48, 16, 1, 1}, {16, 3, 1, 0}};
enum { L_E0A, L_E0B, L_D1, L_E1, L_D2, L_E2, L_D3, L_E3, L_U2, L_U1, L_U0, L_OUT };

inline int cpad4(int c) { return (c + 3) & ~3; }

int fail(int code, const std::string& msg) {
    gmg::set_error_text(msg);
    return code;
}

#define CU(expr)                                                                                               \
    do {                                                                                                       \
        cudaError_t e_ = (expr);                                                                               \
        if (e_ != cudaSuccess) return fail(GMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != GMG_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------ kernels

struct ConvArgs {
    const float* in;
    int in_pitch, cin;
    float* out;
    int out_pitch, cout;      // channels written: [0, cout)
    const float* W;           // [cin][27][w_co]
    int w_co;
    const float* bias;        // [>= cout] or null
    const float* ref;         // activation output whose derivative multiplies (mode 2)
    int ref_pitch;
    int mode;                 // 0 = linear, 1 = leaky ReLU, 2 = times lrelu'(ref)
    int accumulate;           // add the previous content of out
    int X, Y, Z, Xo, Yo, Zo;  // input / output vertex grids
    long long in_bs, out_bs, ref_bs;  // per-sample strides (floats)
    int ci_hi;                // input channels of this launch's split: [blockIdx.z / B * (ci_hi), ...) -- see k_conv
    long long split_bs;       // output stride between input-channel splits (floats)
};

__device__ __forceinline__ float epilogue(float v, const ConvArgs& a, const float* o, long long ridx, int mode) {
    if (a.accumulate) v += *o;
    if (mode == 1) v = v > 0.f ? v : kSlope * v;
    else if (mode == 2) v *= a.ref[ridx] > 0.f ? 1.f : kSlope;
    return v;
}

template <int COB, int TY, int TZ, int S>
struct ConvGeom {
    static constexpr int TX = 8, KC = 4;
    static constexpr int NT = TY * TZ * (COB / 4);
    static constexpr int HX = S * (TX - 1) + 3, HY = S * (TY - 1) + 3, HZ = S * (TZ - 1) + 3;
    static constexpr int HXP = HX | 1;  // odd x pitch: rows of different lanes fall in different banks
    static constexpr int HPLANE = HZ * HY * HXP;
    static constexpr int SMEM_FLOATS = KC * HPLANE + KC * 27 * COB;
    static constexpr size_t SMEM = sizeof(float) * SMEM_FLOATS;
};

template <int COB, int TY, int TZ, int S>
__global__ void __launch_bounds__(ConvGeom<COB, TY, TZ, S>::NT) k_conv(ConvArgs a) {
    using G = ConvGeom<COB, TY, TZ, S>;
    extern __shared__ __align__(16) float smem[];
    float* ws = smem;                      // [KC][27][COB]
    float* hs = smem + G::KC * 27 * COB;   // [KC][HZ][HY][HXP]
    const int tid = threadIdx.x;
    const int row = tid % (TY * TZ);
    const int cg = tid / (TY * TZ);
    const int ty = row % TY, tz = row / TY;
    const int ntx = (a.Xo + G::TX - 1) / G::TX, nty = (a.Yo + TY - 1) / TY;
    int t = blockIdx.x;
    const int bx = t % ntx;
    t /= ntx;
    const int by = t % nty, bz = t / nty;
    const int ox0 = bx * G::TX, oy0 = by * TY, oz0 = bz * TZ;
    const int cob0 = blockIdx.y * COB;
    // blockIdx.z = split * B + b: split k sums input channels [k ci_hi, (k+1) ci_hi)
    // into its own output slice (split_bs apart); ci_hi = cin without a split
    const int nb = a.split_bs ? (int)(gridDim.z / (a.cin / a.ci_hi)) : (int)gridDim.z;
    const int b = blockIdx.z % nb, split = blockIdx.z / nb;
    const float* in = a.in + b * a.in_bs;
    const int ix0 = S * ox0 - 1, iy0 = S * oy0 - 1, iz0 = S * oz0 - 1;

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    const int ci_begin = split * a.ci_hi, ci_end = ci_begin + a.ci_hi;
    for (int ci0 = ci_begin; ci0 < ci_end; ci0 += G::KC) {
        __syncthreads();
        for (int h = tid; h < G::HZ * G::HY * G::HX; h += G::NT) {
            const int hx = h % G::HX;
            const int r = h / G::HX;
            const int hy = r % G::HY, hz = r / G::HY;
            const int ix = ix0 + hx, iy = iy0 + hy, iz = iz0 + hz;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ix >= 0 && ix < a.X && iy >= 0 && iy < a.Y && iz >= 0 && iz < a.Z)
                v = __ldg(reinterpret_cast<const float4*>(in + ((long long)(iz * a.Y + iy) * a.X + ix) * a.in_pitch + ci0));
            const int base = (hz * G::HY + hy) * G::HXP + hx;
            hs[base] = v.x;
            hs[G::HPLANE + base] = v.y;
            hs[2 * G::HPLANE + base] = v.z;
            hs[3 * G::HPLANE + base] = v.w;
        }
        for (int e = tid; e < G::KC * 27 * (COB / 4); e += G::NT) {
            const int j4 = e % (COB / 4);
            const int r = e / (COB / 4);  // c * 27 + tap
            const int co = cob0 + 4 * j4;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (co < a.w_co)
                w = __ldg(reinterpret_cast<const float4*>(a.W + ((long long)(ci0 + r / 27) * 27 + r % 27) * a.w_co + co));
            reinterpret_cast<float4*>(ws)[e] = w;
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < G::KC; ++c) {
#pragma unroll 1
            for (int dz = 0; dz < 3; ++dz) {
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const float* hrow = hs + c * G::HPLANE + ((S * tz + dz) * G::HY + (S * ty + dy)) * G::HXP;
                    float v[G::HX];
#pragma unroll
                    for (int k = 0; k < G::HX; ++k) v[k] = hrow[k];
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const float4 w = reinterpret_cast<const float4*>(ws)[(c * 27 + dx + 3 * dy + 9 * dz) * (COB / 4) + cg];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float xv = v[S * i + dx];
                            acc[i][0] = fmaf(xv, w.x, acc[i][0]);
                            acc[i][1] = fmaf(xv, w.y, acc[i][1]);
                            acc[i][2] = fmaf(xv, w.z, acc[i][2]);
                            acc[i][3] = fmaf(xv, w.w, acc[i][3]);
                        }
                    }
                }
            }
        }
    }

    const int oy = oy0 + ty, oz = oz0 + tz;
    if (oy >= a.Yo || oz >= a.Zo) return;
    const int co = cob0 + 4 * cg;
    if (co >= a.cout) return;
    float bv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = (a.bias && co + j < a.cout) ? a.bias[co + j] : 0.f;
    const bool vec = (co + 4 <= a.cout) && (a.out_pitch % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(a.out) & 15) == 0) && !a.accumulate && a.mode != 2;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int ox = ox0 + i;
        if (ox >= a.Xo) break;
        const long long node = (long long)(oz * a.Yo + oy) * a.Xo + ox;
        float* o = a.out + split * a.split_bs + b * a.out_bs + node * a.out_pitch + co;
        if (vec) {
            float4 r;
            r.x = epilogue(acc[i][0] + bv[0], a, o, 0, a.mode);
            r.y = epilogue(acc[i][1] + bv[1], a, o, 0, a.mode);
            r.z = epilogue(acc[i][2] + bv[2], a, o, 0, a.mode);
            r.w = epilogue(acc[i][3] + bv[3], a, o, 0, a.mode);
            *reinterpret_cast<float4*>(o) = r;
        } else {
            const long long ridx = b * a.ref_bs + node * a.ref_pitch + co;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (co + j < a.cout) o[j] = epilogue(acc[i][j] + bv[j], a, o + j, ridx + j, a.mode);
        }
    }
}

// Backward data pass of a stride-2 layer: g_in[i][ci] = sum over (o, co) with
// i = 2o + d - 1 of W[co][d][ci] g_out[o][co].
struct S2tArgs {
    const float* go;
    int go_pitch, cout;       // cout: multiple of 4
    const float* W;           // [cout][27][cin] (unflipped, rounded)
    int cin;
    float* out;
    int out_pitch;
    const float* ref;
    int ref_pitch;
    int accumulate, mode;     // mode 2: times lrelu'(ref)
    int X, Y, Z, Xo, Yo, Zo;  // fine (input of the layer) / coarse grids
    long long go_bs, out_bs, ref_bs;
};

// A block covers TY x TZ fine rows (y, z) of 8 nodes in x, for all CIG groups of
// 4 input channels.  Threads are ordered parity class (fy & 1) + 2 (fz & 1)
// first, then channel group, then row within the class: TY and TZ are even, so
// every warp holds rows of one class only and never splits over the 1 / 2 / 4
// (y, z) tap combinations of different parities.
template <int CIG>
__global__ void __launch_bounds__(256) k_conv_s2t(S2tArgs a) {
    constexpr int ROWS = 256 / CIG;
    constexpr int TY = ROWS >= 32 ? 8 : 4;
    constexpr int TZ = ROWS / TY;
    constexpr int RPC = ROWS / 4;  // rows per parity class (16, 8, 4: divides 32)
    static_assert(TY % 2 == 0 && TZ % 2 == 0 && 32 % RPC == 0, "parity-major thread order");
    const int tid = threadIdx.x;
    const int cls = tid / (RPC * CIG), cg = (tid / RPC) % CIG, q = tid % RPC;
    const int ty = 2 * (q % (TY / 2)) + (cls & 1), tz = 2 * (q / (TY / 2)) + (cls >> 1);
    const int ntx = (a.X + 7) / 8, nty = (a.Y + TY - 1) / TY;
    int t = blockIdx.x;
    const int bx = t % ntx;
    t /= ntx;
    const int by = t % nty, bz = t / nty;
    const int fx0 = bx * 8, fy = by * TY + ty, fz = bz * TZ + tz;
    const int b = blockIdx.z;
    if (fy >= a.Y || fz >= a.Z) return;
    int dys[2], oys[2], dzs[2], ozs[2];
    int nyy, nzz;
    if ((fy & 1) == 0) { dys[0] = 1; oys[0] = fy >> 1; nyy = 1; }
    else { dys[0] = 0; oys[0] = (fy + 1) >> 1; dys[1] = 2; oys[1] = (fy - 1) >> 1; nyy = 2; }
    if ((fz & 1) == 0) { dzs[0] = 1; ozs[0] = fz >> 1; nzz = 1; }
    else { dzs[0] = 0; ozs[0] = (fz + 1) >> 1; dzs[1] = 2; ozs[1] = (fz - 1) >> 1; nzz = 2; }
    const int oxc = fx0 >> 1;
    const int ci = 4 * cg;
    const float* go = a.go + b * a.go_bs;

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int iz = 0; iz < nzz; ++iz)
        for (int iy = 0; iy < nyy; ++iy) {
            const int tapyz = 3 * dys[iy] + 9 * dzs[iz];
            const float* grow = go + (long long)(ozs[iz] * a.Yo + oys[iy]) * a.Xo * a.go_pitch;
            for (int co0 = 0; co0 < a.cout; co0 += 4) {
                float4 g[5];
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    g[k] = (oxc + k < a.Xo) ? __ldg(reinterpret_cast<const float4*>(grow + (long long)(oxc + k) * a.go_pitch + co0))
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 w[3][4];
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        w[dx][j] = __ldg(reinterpret_cast<const float4*>(a.W + ((long long)(co0 + j) * 27 + tapyz + dx) * a.cin + ci));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if ((k & 1) == 0 && e == 1) continue;
                        const int o = (k & 1) == 0 ? (k >> 1) : (e == 0 ? (k + 1) >> 1 : (k - 1) >> 1);
                        const int dx = (k & 1) == 0 ? 1 : (e == 0 ? 0 : 2);
                        const float gv[4] = {g[o].x, g[o].y, g[o].z, g[o].w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[k][0] = fmaf(gv[j], w[dx][j].x, acc[k][0]);
                            acc[k][1] = fmaf(gv[j], w[dx][j].y, acc[k][1]);
                            acc[k][2] = fmaf(gv[j], w[dx][j].z, acc[k][2]);
                            acc[k][3] = fmaf(gv[j], w[dx][j].w, acc[k][3]);
                        }
                    }
                }
            }
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int fx = fx0 + k;
        if (fx >= a.X) break;
        const long long node = (long long)(fz * a.Y + fy) * a.X + fx;
        float* o = a.out + b * a.out_bs + node * a.out_pitch + ci;
        const float* r = a.ref ? a.ref + b * a.ref_bs + node * a.ref_pitch + ci : nullptr;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = acc[k][j];
            if (a.accumulate) v += o[j];
            if (a.mode == 2) v *= r[j] > 0.f ? 1.f : kSlope;
            o[j] = v;
        }
    }
}

// Weight / bias gradient partial sums over a split of the batch's output nodes.
struct WgArgs {
    const float* in;
    int in_pitch, cin;
    const float* go;
    int go_pitch, coutp;
    int X, Y, Z, Xo, Yo, Zo, B;
    long long in_bs, go_bs;
    long long nodes_per_split;
    float* part;              // [splits][coutp*27*cin + coutp]
    long long part_stride;
};

// One thread per (4 output channels, 4 input channels, tap row (dy, dz)); it
// holds the three taps dx = 0, 1, 2 of the row, so each node costs one load of
// the output gradient and three of the input (neighbours in x) for 48 FMAs.
template <int S>
__global__ void __launch_bounds__(256) k_wgrad(WgArgs a) {
    const int cin4 = a.cin / 4;
    const int pairs = (a.coutp / 4) * cin4;
    const int task = blockIdx.y * 256 + threadIdx.x;
    if (task >= pairs * 9) return;
    const int trow = task / pairs, pr = task % pairs;
    const int ci4 = pr % cin4, co4 = pr / cin4;
    const int dy = trow % 3, dz = trow / 3;
    const long long No = (long long)a.Xo * a.Yo * a.Zo;
    const long long o_begin = blockIdx.x * a.nodes_per_split;
    const long long o_end = min(o_begin + a.nodes_per_split, No * a.B);
    float acc[3][4][4];
    float bacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[d][j][k] = 0.f;
    const bool do_bias = (trow == 4) && (ci4 == 0);  // the row holding the centre tap 13
    if (o_begin < o_end) {
        long long r = o_begin;
        int b = (int)(r / No);
        long long on = r - (long long)b * No;
        int ox = (int)(on % a.Xo);
        int oy = (int)((on / a.Xo) % a.Yo);
        int oz = (int)(on / ((long long)a.Xo * a.Yo));
        for (long long o = o_begin; o < o_end; ++o) {
            const float4 g = __ldg(reinterpret_cast<const float4*>(a.go + b * a.go_bs + on * a.go_pitch + 4 * co4));
            const int iy = S * oy + dy - 1, iz = S * oz + dz - 1;
            if (iy >= 0 && iy < a.Y && iz >= 0 && iz < a.Z) {
                const float* xrow = a.in + b * a.in_bs + ((long long)(iz * a.Y + iy) * a.X) * a.in_pitch + 4 * ci4;
                const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int ix = S * ox + dx - 1;
                    if (ix >= 0 && ix < a.X) {
                        const float4 x = __ldg(reinterpret_cast<const float4*>(xrow + (long long)ix * a.in_pitch));
                        const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int k = 0; k < 4; ++k) acc[dx][j][k] = fmaf(gv[j], xv[k], acc[dx][j][k]);
                    }
                }
            }
            if (do_bias) {
                bacc[0] += g.x;
                bacc[1] += g.y;
                bacc[2] += g.z;
                bacc[3] += g.w;
            }
            ++on;
            if (++ox == a.Xo) {
                ox = 0;
                if (++oy == a.Yo) {
                    oy = 0;
                    if (++oz == a.Zo) {
                        oz = 0;
                        ++b;
                        on = 0;
                    }
                }
            }
        }
    }
    float* p = a.part + blockIdx.x * a.part_stride;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
        const int tap = dx + 3 * trow;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) p[((long long)(4 * co4 + j) * 27 + tap) * a.cin + 4 * ci4 + k] = acc[dx][j][k];
    }
    if (do_bias)
#pragma unroll
        for (int j = 0; j < 4; ++j) p[(long long)a.coutp * 27 * a.cin + 4 * co4 + j] = bacc[j];
}

// Input-channel splits of a convolution: out[node][co] = act(bias + sum over
// splits of part[k][node][co]) in split order (part has pitch cout).
__global__ void k_split_sum(const float* __restrict__ part, int splits, long long split_bs, long long nodes, int cout,
                            const float* __restrict__ bias, int act, float* __restrict__ out, int out_pitch,
                            long long out_bs, long long nodes_per_sample) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nodes * cout) return;
    const long long n = i / cout;
    const int co = (int)(i % cout);
    float v = 0.f;
    for (int k = 0; k < splits; ++k) v += part[k * split_bs + i];
    v += bias[co];
    if (act) v = v > 0.f ? v : kSlope * v;
    const long long b = n / nodes_per_sample, nl = n % nodes_per_sample;
    out[b * out_bs + nl * out_pitch + co] = v;
}

// out[i] = sum_s part[s * stride + i] in split order.
__global__ void k_sum_splits(const float* __restrict__ part, long long stride, int splits, long long n,
                             float* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[k * stride + i];
    out[i] = s;
}

// Trilinear (vertex-centred) prolongation of C channels from the coarse grid
// (Xc, Yc, Zc) into out (fine grid 2Xc-1 ..., pitch po, C channels written).
__global__ void k_upsample(const float* __restrict__ in, int pi, float* __restrict__ out, int po, int C, int Xc,
                           int Yc, int Zc, long long in_bs, long long out_bs, int B) {
    const int X = 2 * Xc - 1, Y = 2 * Yc - 1, Z = 2 * Zc - 1;
    const int C4 = C / 4;
    const long long n = (long long)X * Y * Z * C4 * B;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c4 = (int)(idx % C4);
    long long r = idx / C4;
    const int i = (int)(r % X);
    r /= X;
    const int j = (int)(r % Y);
    r /= Y;
    const int k = (int)(r % Z);
    const int b = (int)(r / Z);
    const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1, k1 = (k + 1) >> 1;
    const float wi1 = (i & 1) ? 0.5f : 0.f, wj1 = (j & 1) ? 0.5f : 0.f, wk1 = (k & 1) ? 0.5f : 0.f;
    const float wi[2] = {1.f - wi1, wi1}, wj[2] = {1.f - wj1, wj1}, wk[2] = {1.f - wk1, wk1};
    const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* src = in + b * in_bs + 4 * c4;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int aa = 0; aa < 2; ++aa) {
                const float w = wk[c] * wj[bb] * wi[aa];
                if (w == 0.f) continue;
                const float4 v = __ldg(reinterpret_cast<const float4*>(src + ((long long)(kk[c] * Yc + jj[bb]) * Xc + ii[aa]) * pi));
                s.x = fmaf(w, v.x, s.x);
                s.y = fmaf(w, v.y, s.y);
                s.z = fmaf(w, v.z, s.z);
                s.w = fmaf(w, v.w, s.w);
            }
    *reinterpret_cast<float4*>(out + b * out_bs + ((long long)(k * Y + j) * X + i) * po + 4 * c4) = s;
}

// Adjoint of k_upsample, times the leaky-ReLU derivative of ref (coarse).
__global__ void k_upsample_adj(const float* __restrict__ g, int pg, float* __restrict__ out, int po,
                               const float* __restrict__ ref, int pr, int C, int Xc, int Yc, int Zc, long long g_bs,
                               long long out_bs, long long ref_bs, int B) {
    const int X = 2 * Xc - 1, Y = 2 * Yc - 1, Z = 2 * Zc - 1;
    const int C4 = C / 4;
    const long long n = (long long)Xc * Yc * Zc * C4 * B;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c4 = (int)(idx % C4);
    long long r = idx / C4;
    const int I = (int)(r % Xc);
    r /= Xc;
    const int J = (int)(r % Yc);
    r /= Yc;
    const int K = (int)(r % Zc);
    const int b = (int)(r / Zc);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* src = g + b * g_bs + 4 * c4;
    for (int dk = -1; dk <= 1; ++dk) {
        const int k = 2 * K + dk;
        if (k < 0 || k >= Z) continue;
        const float wk = dk == 0 ? 1.f : 0.5f;
        for (int dj = -1; dj <= 1; ++dj) {
            const int j = 2 * J + dj;
            if (j < 0 || j >= Y) continue;
            const float wj = dj == 0 ? 1.f : 0.5f;
            for (int di = -1; di <= 1; ++di) {
                const int i = 2 * I + di;
                if (i < 0 || i >= X) continue;
                const float w = wk * wj * (di == 0 ? 1.f : 0.5f);
                const float4 v = __ldg(reinterpret_cast<const float4*>(src + ((long long)(k * Y + j) * X + i) * pg));
                s.x = fmaf(w, v.x, s.x);
                s.y = fmaf(w, v.y, s.y);
                s.z = fmaf(w, v.z, s.z);
                s.w = fmaf(w, v.w, s.w);
            }
        }
    }
    const long long node = (long long)(K * Yc + J) * Xc + I;
    const float4 rv = __ldg(reinterpret_cast<const float4*>(ref + b * ref_bs + node * pr + 4 * c4));
    s.x *= rv.x > 0.f ? 1.f : kSlope;
    s.y *= rv.y > 0.f ? 1.f : kSlope;
    s.z *= rv.z > 0.f ? 1.f : kSlope;
    s.w *= rv.w > 0.f ? 1.f : kSlope;
    *reinterpret_cast<float4*>(out + b * out_bs + node * po + 4 * c4) = s;
}

// Fixed-order reduction over the 256 threads of a block (sum, or max with
// op = 1); every thread gets the result.  Deterministic: thread t first folds
// partials t, t + 256, ... in order, then the tree has a fixed shape.
template <int OP>
__device__ double block_reduce256(double v) {
    __shared__ double sh[256];
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) sh[t] = OP == 0 ? sh[t] + sh[t + w] : fmax(sh[t], sh[t + w]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double fold(const double* p, int n, int stride, int off, int op) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) v = op == 0 ? v + p[(long long)i * stride + off] : fmax(v, p[(long long)i * stride + off]);
    return v;
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 296;  // 2 x 148 SMs

// partial[block] = number of nodes (over the batch) whose feature channel 4 < 0.5
__global__ void __launch_bounds__(kRedThreads) k_count_free(const float* __restrict__ x, long long nodes, double* partial) {
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (long long n = blockIdx.x * (long long)kRedThreads + threadIdx.x; n < nodes; n += (long long)gridDim.x * kRedThreads)
        s += x[n * GMG_NET_IN + 4] < 0.5f ? 1.0 : 0.0;
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// sc[slot] = scale * sum(partial[0..n))
__global__ void __launch_bounds__(256) k_finish_sum(const double* partial, int n, double scale, double* sc, int slot) {
    const double s = block_reduce256<0>(fold(partial, n, 1, 0, 0));
    if (threadIdx.x == 0) sc[slot] = scale * s;
}

// gg = 2 (g - t) mask / count on channels 0..2 (channel 3 = 0); partial sums of (g - t)^2 mask.
__global__ void __launch_bounds__(kRedThreads) k_loss(const float* __restrict__ g, const float* __restrict__ t,
                                                      const float* __restrict__ x, long long nodes,
                                                      const double* __restrict__ sc, float* __restrict__ gg,
                                                      double* partial) {
    __shared__ double sh[kRedThreads];
    const float scale = sc[0] > 0.0 ? (float)(2.0 / sc[0]) : 0.f;
    double s = 0.0;
    for (long long n = blockIdx.x * (long long)kRedThreads + threadIdx.x; n < nodes; n += (long long)gridDim.x * kRedThreads) {
        const float m = x[n * GMG_NET_IN + 4] < 0.5f ? 1.f : 0.f;
        float4 o;
        const float4 gv = *reinterpret_cast<const float4*>(g + 4 * n);
        const float d0 = (gv.x - t[3 * n]) * m, d1 = (gv.y - t[3 * n + 1]) * m, d2 = (gv.z - t[3 * n + 2]) * m;
        s += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2;
        o.x = scale * d0;
        o.y = scale * d1;
        o.z = scale * d2;
        o.w = 0.f;
        *reinterpret_cast<float4*>(gg + 4 * n) = o;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// loss = sum(partial) / count, as float
__global__ void __launch_bounds__(256) k_loss_finish(const double* partial, int n, const double* sc, float* loss) {
    const double s = block_reduce256<0>(fold(partial, n, 1, 0, 0));
    if (threadIdx.x == 0) *loss = sc[0] > 0.0 ? (float)(s / sc[0]) : 0.f;
}

// Energy loss, step 1: gm = g and tm = t on the free DOFs (0 on fixed ones)
// for B samples; g has pitch 4, t pitch 3, mask = per-node fixed-component bits.
__global__ void k_energy_prep(const float* __restrict__ g, const float* __restrict__ t, const uint8_t* __restrict__ mask,
                              long long nn, int B, float* __restrict__ gm, float* __restrict__ tm) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 3 * nn * B) return;
    const long long bn = i / 3;  // b * nn + n
    const int c = (int)(i % 3);
    const bool fx = (mask[bn] >> c) & 1;
    gm[i] = fx ? 0.f : g[4 * bn + c];
    tm[i] = fx ? 0.f : t[i];
}

constexpr int kEnergyBlocks = 64;  // reduction blocks per sample

// Per sample b (blockIdx.y): partial[(b * kEnergyBlocks + block) * 3 + {0,1,2}] =
// sums of tm.Kg, gm.Kg, tm.Kt over that sample's n = 3 nn entries.
__global__ void __launch_bounds__(kRedThreads) k_energy_dots(const float* __restrict__ gm, const float* __restrict__ kg,
                                                             const float* __restrict__ tm, const float* __restrict__ kt,
                                                             long long n, double* partial) {
    __shared__ double sh[3][kRedThreads];
    const long long off = blockIdx.y * n;
    double a = 0.0, b = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kRedThreads) {
        const double t = tm[off + i], g = gm[off + i], Kg = kg[off + i];
        a += t * Kg;
        b += g * Kg;
        c += t * (double)kt[off + i];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 3 + k] = sh[k][0];
}

// Per sample: L_b = 1 - a^2 / (b c); dL/dg_b = coef[2b] K g + coef[2b+1] K t with
// coef = (2a/(bc)) (a/b, -1) / B (zero, and L_b = 1, when b or c is not positive).
// loss = mean of L_b.
__global__ void __launch_bounds__(256) k_energy_finish(const double* partial, int nb, int B, double* coef, float* loss) {
    double L = 0.0;
    for (int s = 0; s < B; ++s) {
        const double* ps = partial + (long long)s * nb * 3;
        const double a = block_reduce256<0>(fold(ps, nb, 3, 0, 0));
        const double b = block_reduce256<0>(fold(ps, nb, 3, 1, 0));
        const double c = block_reduce256<0>(fold(ps, nb, 3, 2, 0));
        if (threadIdx.x != 0) continue;
        if (b > 0.0 && c > 0.0 && isfinite(a) && isfinite(b) && isfinite(c)) {
            L += 1.0 - a * a / (b * c);
            const double k = 2.0 * a / (b * c) / (double)B;
            coef[2 * s] = k * a / b;
            coef[2 * s + 1] = -k;
        } else {
            L += 1.0;
            coef[2 * s] = 0.0;
            coef[2 * s + 1] = 0.0;
        }
    }
    if (threadIdx.x == 0) *loss = (float)(L / (double)B);
}

// gg[b][n][c] = coef[2b] Kg + coef[2b+1] Kt (pitch 4, channel 3 = 0)
__global__ void k_energy_grad(const float* __restrict__ kg, const float* __restrict__ kt, long long nn, int B,
                              const double* __restrict__ coef, float* __restrict__ gg) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= nn * B) return;
    const int b = (int)(n / nn);
    const float s1 = (float)coef[2 * b], s2 = (float)coef[2 * b + 1];
    float4 o;
    o.x = s1 * kg[3 * n] + s2 * kt[3 * n];
    o.y = s1 * kg[3 * n + 1] + s2 * kt[3 * n + 1];
    o.z = s1 * kg[3 * n + 2] + s2 * kt[3 * n + 2];
    o.w = 0.f;
    *reinterpret_cast<float4*>(gg + 4 * n) = o;
}

struct LayerTable {
    long long woff[kLayers], boff[kLayers];
    int cin[kLayers], coutp[kLayers];
};

// partial[block] = sum of squares of a float vector
__global__ void __launch_bounds__(kRedThreads) k_sumsq_f(const float* __restrict__ v, long long n, double* partial) {
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kRedThreads)
        s += (double)v[i] * (double)v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Adam step counter, bias corrections and gradient scale: adam[0] = t,
// adam[1] = 1/(1-b1^t), adam[2] = 1/(1-b2^t), adam[3] = min(1, clip/|g|)
// (1 without clipping, 0 for a non-finite norm).
__global__ void __launch_bounds__(256) k_adam_tick(double* adam, const double* gnorm_partial, int nb, const float* clip) {
    const double ss = block_reduce256<0>(fold(gnorm_partial, nb, 1, 0, 0));
    if (threadIdx.x != 0) return;
    const double t = adam[0] + 1.0;
    adam[0] = t;
    adam[1] = 1.0 / (1.0 - pow(kBeta1, t));
    adam[2] = 1.0 / (1.0 - pow(kBeta2, t));
    const double nrm = sqrt(ss);
    const double c = (double)clip[0];
    double scale = 1.0;
    if (!isfinite(nrm)) scale = 0.0;
    else if (c > 0.0 && nrm > c) scale = c / nrm;
    adam[3] = scale;
}

// Writes the bfloat16-rounded copies of weight i of layer l: Wr (own layout),
// Wf [cin][27][coutp] (forward) and Wb [coutp][26-tap][cin] (backward data).
__device__ __forceinline__ void scatter_weight(const LayerTable& T, int l, long long j, float w, float* Wr, float* Wf,
                                               float* Wb) {
    const int cin = T.cin[l], coutp = T.coutp[l];
    const int ci = (int)(j % cin);
    const int tap = (int)((j / cin) % 27);
    const int co = (int)(j / (27LL * cin));
    const float r = __bfloat162float(__float2bfloat16_rn(w));
    const long long base = T.woff[l];
    Wr[base + j] = r;
    Wf[base + ((long long)ci * 27 + tap) * coutp + co] = r;
    Wb[base + ((long long)co * 27 + (26 - tap)) * cin + ci] = r;
}

__device__ __forceinline__ int layer_of(const LayerTable& T, long long i) {
    int l = 0;
    while (l + 1 < kLayers && i >= T.woff[l + 1]) ++l;
    return l;
}

__global__ void k_adam(const LayerTable T, long long n, float* __restrict__ P, float* __restrict__ M,
                       float* __restrict__ V, const float* __restrict__ G, float* __restrict__ Wr,
                       float* __restrict__ Wf, float* __restrict__ Wb, const double* __restrict__ adam,
                       const float* __restrict__ lr) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c1 = (float)adam[1], c2 = (float)adam[2];
    const float g = G[i] * (float)adam[3];
    const float m = (float)kBeta1 * M[i] + (1.f - (float)kBeta1) * g;
    const float v = (float)kBeta2 * V[i] + (1.f - (float)kBeta2) * g * g;
    M[i] = m;
    V[i] = v;
    const float w = P[i] - lr[0] * (m * c1) / (sqrtf(v * c2) + (float)kAdamEps);
    P[i] = w;
    const int l = layer_of(T, i);
    if (i < T.boff[l]) scatter_weight(T, l, i - T.woff[l], w, Wr, Wf, Wb);
    else Wr[i] = w;
}

// Rounded copies of all weights from the master parameters (after set_params).
__global__ void k_round_all(const LayerTable T, long long n, const float* __restrict__ P, float* __restrict__ Wr,
                            float* __restrict__ Wf, float* __restrict__ Wb) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = layer_of(T, i);
    if (i < T.boff[l]) scatter_weight(T, l, i - T.woff[l], P[i], Wr, Wf, Wb);
    else Wr[i] = P[i];
}

// Load statistics of one problem: partial[4 block + 0] = max |f|,
// partial[4 block + 1..3] = sum of the x / y / z load components.
__global__ void __launch_bounds__(kRedThreads) k_load_stats(const double* __restrict__ f, long long nn, double* partial) {
    __shared__ double sh[4][kRedThreads];
    double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (long long n = blockIdx.x * (long long)kRedThreads + threadIdx.x; n < nn; n += (long long)gridDim.x * kRedThreads) {
        const double a = f[3 * n], b = f[3 * n + 1], c = f[3 * n + 2];
        m = fmax(m, fmax(fabs(a), fmax(fabs(b), fabs(c))));
        sx += a;
        sy += b;
        sz += c;
    }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = sx;
    sh[2][threadIdx.x] = sy;
    sh[3][threadIdx.x] = sz;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + w]);
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] += sh[3][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partial[4 * blockIdx.x + k] = sh[k][0];
}

// stats[0] = 1 / max|f| (0 for f = 0), stats[1..3] = sum(f) / |sum(f)| (0 when it vanishes)
__global__ void __launch_bounds__(256) k_load_stats_finish(const double* partial, int nb, double* stats) {
    const double m = block_reduce256<1>(fold(partial, nb, 4, 0, 1));
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = block_reduce256<0>(fold(partial, nb, 4, 1 + k, 0));
    if (threadIdx.x != 0) return;
    stats[0] = m > 0.0 ? 1.0 / m : 0.0;
    const double r = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) stats[1 + k] = r > 0.0 ? s[k] / r : 0.0;
}

// Input features of one problem (see gmg_warmnet.h).  Exactly one of fixed
// (per-DOF flags) and mask (per-node component bits) is non-null.
__global__ void k_features(int nx, int ny, int nz, const float* __restrict__ rho, const double* __restrict__ f,
                           const uint8_t* __restrict__ fixed, const uint8_t* __restrict__ mask,
                           const double* __restrict__ stats, float* __restrict__ x) {
    const int X = nx + 1, Y = ny + 1, Z = nz + 1;
    const long long nn = (long long)X * Y * Z;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const int i = (int)(n % X), j = (int)((n / X) % Y), k = (int)(n / ((long long)X * Y));
    float s = 0.f, c = 0.f;
    for (int ez = k - 1; ez <= k; ++ez)
        for (int ey = j - 1; ey <= j; ++ey)
            for (int ex = i - 1; ex <= i; ++ex)
                if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz) {
                    s += rho[((long long)ez * ny + ey) * nx + ex];
                    c += 1.f;
                }
    const double inv = stats[0];
    bool fx;
    if (fixed) fx = fixed[3 * n] | fixed[3 * n + 1] | fixed[3 * n + 2];
    else fx = mask[n] != 0;
    float4 a, bq, cq;
    a.x = s / c;
    a.y = (float)(f[3 * n] * inv);
    a.z = (float)(f[3 * n + 1] * inv);
    a.w = (float)(f[3 * n + 2] * inv);
    bq.x = fx ? 1.f : 0.f;
    bq.y = (float)i / (float)nx;
    bq.z = (float)j / (float)ny;
    bq.w = (float)k / (float)nz;
    cq.x = (float)stats[1];
    cq.y = (float)stats[2];
    cq.z = (float)stats[3];
    cq.w = 1.f;
    float4* o = reinterpret_cast<float4*>(x + GMG_NET_IN * n);
    o[0] = a;
    o[1] = bq;
    o[2] = cq;
}

// partial[block] = max |v| (kind 0) or sum v^2 (kind 1) over a double vector.
__global__ void __launch_bounds__(kRedThreads) k_reduce_vec(const double* __restrict__ v, long long n, int kind,
                                                            double* partial) {
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kRedThreads)
        s = kind == 0 ? fmax(s, fabs(v[i])) : s + v[i] * v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = kind == 0 ? fmax(sh[threadIdx.x], sh[threadIdx.x + w]) : sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) k_finish_vec(const double* partial, int n, int kind, double* out) {
    const double s = kind == 0 ? block_reduce256<1>(fold(partial, n, 1, 0, 1)) : block_reduce256<0>(fold(partial, n, 1, 0, 0));
    if (threadIdx.x == 0) *out = s;
}

// t = u / sqrt(sumsq / n)   (0 when u = 0)
__global__ void k_target(const double* __restrict__ u, long long n, const double* __restrict__ sumsq, float* __restrict__ t) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ss = sumsq[0];
    const double inv = ss > 0.0 ? 1.0 / sqrt(ss / (double)n) : 0.0;
    t[i] = (float)(u[i] * inv);
}

// gd[3n + c] = g[4n + c] masked by the node's fixed-component bits
__global__ void k_out_to_dofs(const float* __restrict__ g, const uint8_t* __restrict__ mask, long long nn,
                              float* __restrict__ gd) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 3 * nn) return;
    const long long n = i / 3;
    const int c = (int)(i % 3);
    gd[i] = ((mask[n] >> c) & 1) ? 0.f : g[4 * n + c];
}

// partial[2 block + 0] = sum f.g, partial[2 block + 1] = sum g.Kg
__global__ void __launch_bounds__(kRedThreads) k_ws_dots(const double* __restrict__ f, const float* __restrict__ g,
                                                         const float* __restrict__ kg, long long n, double* partial) {
    __shared__ double sa[kRedThreads], sb[kRedThreads];
    double a = 0.0, b = 0.0;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kRedThreads) {
        a += f[i] * (double)g[i];
        b += (double)g[i] * (double)kg[i];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sa[0];
        partial[2 * blockIdx.x + 1] = sb[0];
    }
}

__global__ void __launch_bounds__(256) k_ws_alpha(const double* partial, int nb, double* alpha) {
    const double a = block_reduce256<0>(fold(partial, nb, 2, 0, 0));
    const double b = block_reduce256<0>(fold(partial, nb, 2, 1, 0));
    if (threadIdx.x != 0) return;
    *alpha = (b > 0.0 && isfinite(a) && isfinite(b)) ? a / b : 0.0;
}

__global__ void k_ws_scale(const float* __restrict__ g, long long n, const double* __restrict__ alpha, double* __restrict__ u0) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    u0[i] = alpha[0] * (double)g[i];
}

// ---------------------------------------------------------------------------
// Tensor-core convolution, stride 1: implicit GEMM on tcgen05 (kind::tf32,
// FP32 accumulation in TMEM).  A CTA owns an 8 (x) x 16 (y) x 1 (z) tile of
// output nodes = M 128 and NB output channels.  Per chunk of 8 input channels
// TMA brings the input halo (10 x 18 x 3 nodes) as two 4-channel slabs laid
// out [z][y][x][4]: eight x-consecutive nodes are one 8-row x 16-byte core
// matrix, the next y row the next 8-row group (160 bytes on), the second slab
// (8,704 bytes on) the next 4 channels of K -- so the A operand of each of the 27 taps is the
// same halo seen through a shifted descriptor, and the halo is loaded once per
// chunk instead of once per tap.  The weights of the chunk (all taps, laid out
// by k_tc_image in the same K-major core-matrix form) come with one bulk copy.
// One thread streams the chunks through two stages and issues the 27 MMAs per
// chunk; all four warps then read the accumulator rows (one output node per
// thread) and apply bias, activation / derivative and the store.  The
// activations stay FP32 in memory; the MMA reads them as TF32, and the
// weights are bfloat16-valued, hence exact in TF32.
// ---------------------------------------------------------------------------
constexpr int kTcHX = 10, kTcHY = 18, kTcHZ = 3;  // halo of an 8 x 16 x 1 output tile
constexpr unsigned kTcSlab = kTcHX * kTcHY * kTcHZ * 16;  // bytes of one 4-channel slab (one TMA box)
constexpr unsigned kTcSlabPitch = (kTcSlab + 127u) & ~127u;  // its stride in shared memory (128-byte aligned)
constexpr unsigned kTcSpinW = 1u << 20;

template <int NB>
struct TcGeom {
    static constexpr unsigned W = 27u * 32u * NB;             // weight bytes of one 8-channel chunk
    static constexpr unsigned STAGE = 2u * kTcSlabPitch + W;  // bytes of one pipeline stage
    static constexpr unsigned TX = 2u * kTcSlab + W;          // bytes the stage's copies deliver
    static constexpr unsigned SMEM = 2u * STAGE + 1024u;
    static constexpr unsigned COLS = NB < 32 ? 32u : (unsigned)NB;
};

struct TcConvArgs {
    float* out;
    int out_pitch, cout;      // channels written: [0, cout)
    const float* img;         // weight image [nblk][nch][27][2][NB/8][8][4]
    const float* bias;
    const float* ref;
    int ref_pitch;
    int mode, accumulate;     // as ConvArgs
    int X, Y, Z;
    int nch;                  // 8-channel chunks of the input
    long long out_bs, ref_bs;
    int* err;
};

__device__ __forceinline__ uint64_t tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    // K-major, no swizzle: lbo = byte distance of K-adjacent core matrices,
    // sbo = byte distance of adjacent 8-row groups
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_tf32(unsigned d, uint64_t da, uint64_t db, unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned addr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NB>
__global__ void __launch_bounds__(128, 1) k_conv_tc(const __grid_constant__ CUtensorMap tm, TcConvArgs a) {
    using Gm = TcGeom<NB>;
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) uint64_t full[2], empty[2], done;
    __shared__ unsigned tslot;
    __shared__ int fail_flag;
    unsigned char* dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);  // 1 KB aligned
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (a.X + 7) >> 3, nty = (a.Y + 15) >> 4;
    int t = blockIdx.x;
    const int bx = t % ntx;
    t /= ntx;
    const int by = t % nty, z = t / nty;
    const int x0 = bx * 8, y0 = by * 16;
    const int nblk = blockIdx.y, b = blockIdx.z;
    if (tid == 0) {
        fail_flag = 0;
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        mbar_init(&done, 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(Gm::COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tslot;

    if (tid == 0) {
        const unsigned base = smem_u32(dyn);
        const float* img = a.img + (size_t)nblk * a.nch * (Gm::W / 4);
        auto wait = [&](uint64_t* bar, unsigned par) -> bool {
            for (unsigned it = 0; it < kTcSpinW; ++it)
                if (mbar_try_wait(bar, par)) return true;
            return false;
        };
        auto load = [&](int c, int st) {
            unsigned char* sp = dyn + st * Gm::STAGE;
            mbar_expect_tx(&full[st], Gm::TX);
            tma_load_5d(sp, &tm, 8 * c, x0 - 1, y0 - 1, z - 1, b, &full[st]);
            tma_load_5d(sp + kTcSlabPitch, &tm, 8 * c + 4, x0 - 1, y0 - 1, z - 1, b, &full[st]);
            bulk_load(sp + 2 * kTcSlabPitch, img + (size_t)c * (Gm::W / 4), Gm::W, &full[st]);
        };
        constexpr unsigned idesc =
            (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NB >> 3) << 17) | ((128u >> 4) << 24);
        bool ok = true;
        int loaded = 0, consumed = 0;
        load(0, 0);
        loaded = 1;
        if (a.nch > 1) {
            load(1, 1);
            loaded = 2;
        }
        for (int c = 0; c < a.nch; ++c) {
            const int st = c & 1;
            if (!wait(&full[st], (c >> 1) & 1)) {
                ok = false;
                break;
            }
            consumed = c + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned ab = base + st * Gm::STAGE, wb = ab + 2 * kTcSlabPitch;
            const uint64_t da0 = tc_desc(ab, kTcSlabPitch, kTcHX * 16), db0 = tc_desc(wb, 16 * NB, 128);
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
                const uint64_t da = da0 + (uint64_t)((((dz * kTcHY + dy) * kTcHX + dx) * 16) >> 4);
                const uint64_t db = db0 + (uint64_t)((tap * 32 * NB) >> 4);
                mma_tf32(tmem, da, db, idesc, (c > 0 || tap > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[st]))
                         : "memory");
            if (c + 2 < a.nch) {
                if (!wait(&empty[st], (c >> 1) & 1)) {
                    ok = false;
                    break;
                }
                load(c + 2, st);
                loaded = c + 3;
            }
        }
        // all MMAs issued so far, then every load still in flight, must finish
        // before the shared memory and TMEM are given up
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
        if (!wait(&done, 0)) ok = false;
        for (int c = consumed; c < loaded; ++c)
            if (!wait(&full[c & 1], (c >> 1) & 1)) ok = false;
        if (!ok) {
            fail_flag = 1;
            atomicExch(a.err, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!fail_flag) {
        float v[NB];
        const unsigned row = tmem + ((unsigned)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < NB; c += 16) tmem_ld16(row + c, v + c);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int m = 32 * warp + lane;
        const int x = x0 + (m & 7), y = y0 + (m >> 3);
        const int co0 = nblk * NB;
        if (x < a.X && y < a.Y) {
            const long long node = (long long)(z * a.Y + y) * a.X + x;
            float* o = a.out + b * a.out_bs + node * a.out_pitch + co0;
            const float* r = a.ref ? a.ref + b * a.ref_bs + node * a.ref_pitch + co0 : nullptr;
            const int nc = min(NB, a.cout - co0);
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j >= nc) break;
                float val = v[j];
                if (a.bias) val += a.bias[co0 + j];
                if (a.accumulate) val += o[j];
                if (a.mode == 1) val = val > 0.f ? val : kSlope * val;
                else if (a.mode == 2) val *= r[j] > 0.f ? 1.f : kSlope;
                o[j] = val;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Gm::COLS) : "memory");
}

// ---------------------------------------------------------------------------
// Tensor-core convolution, stride 1, z-marching: a CTA owns an 8 x 16 tile of
// output nodes over a range of z-planes.  Its weights (every chunk and tap)
// stay in shared memory for the whole range; the input arrives one z-plane at
// a time (all channel slabs of the 10 x 18 halo, one TMA box per 4 channels)
// into a ring of four plane slots, so each plane is loaded once and serves
// the three output planes that read it.  Output plane z takes its 27 taps
// from the slots of planes z-1, z, z+1 through shifted descriptors.  One
// thread (warp 4) issues the loads and the MMAs into two TMEM accumulators
// used alternately; warps 0-3 drain the accumulator of plane z (bias,
// activation, store) while the MMAs of plane z+1 run.
// ---------------------------------------------------------------------------
constexpr unsigned kTczSlab = kTcHX * kTcHY * 16;              // one 4-channel slab of one plane: 2,880 bytes
constexpr unsigned kTczSlabPitch = (kTczSlab + 127u) & ~127u;  // 2,944: 128-byte aligned TMA destinations
constexpr int kTczRing = 4;

struct TczArgs {
    float* out;
    int out_pitch, cout;
    const float* img;   // weight image of one output block: [nch][27][2][NB/8][8][4]
    const float* bias;
    int mode;           // 0 = linear, 1 = leaky ReLU
    int X, Y, Z;
    int nch, nslab;     // 8-channel chunks, 4-channel slabs (2 nch)
    int zr;             // output planes per CTA
    long long out_bs;
    int* err;
};

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int NB>
__global__ void __launch_bounds__(160, 1) k_conv_tcz(const __grid_constant__ CUtensorMap tm, TczArgs a) {
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) uint64_t wbar, pfull[kTczRing], mdone[2], afree[2], fin;
    __shared__ unsigned tslot;
    __shared__ volatile int abort_flag;
    constexpr unsigned COLS = 2 * NB < 32 ? 32u : 2u * NB;  // two accumulators of NB columns
    unsigned char* dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
    const unsigned WB = (unsigned)a.nch * 27u * 32u * NB;
    const unsigned SLOT = (unsigned)a.nslab * kTczSlabPitch;
    unsigned char* wsm = dyn;
    unsigned char* ring = dyn + WB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (a.X + 7) >> 3;
    const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
    const int x0 = bx * 8, y0 = by * 16;
    const int z0 = blockIdx.y * a.zr, z1 = min(z0 + a.zr, a.Z);
    const int nz = z1 - z0, np = nz + 2;
    const int b = blockIdx.z;
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(&wbar, 1);
        for (int i = 0; i < kTczRing; ++i) mbar_init(&pfull[i], 1);
        mbar_init(&mdone[0], 1);
        mbar_init(&mdone[1], 1);
        mbar_init(&afree[0], 128);
        mbar_init(&afree[1], 128);
        mbar_init(&fin, 1);
        mbar_fence_init();
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tslot;

    if (warp == 4) {
        if (lane == 0) {
            auto wait = [&](uint64_t* bar, unsigned par) -> bool {
                for (unsigned it = 0; it < kTcSpinW; ++it) {
                    if (mbar_try_wait(bar, par)) return true;
                    if (abort_flag) return false;
                }
                return false;
            };
            int last_q[kTczRing] = {-1, -1, -1, -1}, seen_q[kTczRing] = {-1, -1, -1, -1};
            auto load_plane = [&](int q) {
                const int slot = q & (kTczRing - 1);
                unsigned char* dst = ring + slot * SLOT;
                mbar_expect_tx(&pfull[slot], (unsigned)a.nslab * kTczSlab);
                for (int sl = 0; sl < a.nslab; ++sl)
                    tma_load_5d(dst + sl * kTczSlabPitch, &tm, 4 * sl, x0 - 1, y0 - 1, z0 - 1 + q, b, &pfull[slot]);
                last_q[slot] = q;
            };
            constexpr unsigned idesc =
                (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NB >> 3) << 17) | ((128u >> 4) << 24);
            const uint64_t da0 = tc_desc(smem_u32(ring), kTczSlabPitch, kTcHX * 16);
            const uint64_t db0 = tc_desc(smem_u32(wsm), 16 * NB, 128);
            mbar_expect_tx(&wbar, WB);
            bulk_load(wsm, a.img, WB, &wbar);
            for (int q = 0; q < kTczRing && q < np; ++q) load_plane(q);
            bool ok = wait(&wbar, 0);
            bool w_seen = ok;
            for (int zi = 0; zi < nz && ok; ++zi) {
                for (int q = zi; q < zi + 3 && ok; ++q) {
                    ok = wait(&pfull[q & (kTczRing - 1)], (q >> 2) & 1);
                    if (ok) seen_q[q & (kTczRing - 1)] = q;
                }
                if (ok && zi >= 2) ok = wait(&afree[zi & 1], ((zi - 2) >> 1) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned acc = tmem + (unsigned)((zi & 1) * NB);
                // descriptors differ from the base ones only in the address
                // field (address / 16), so each tap is a constant offset
                const uint64_t sa[3] = {da0 + (((unsigned)((zi) & (kTczRing - 1)) * SLOT) >> 4),
                                        da0 + (((unsigned)((zi + 1) & (kTczRing - 1)) * SLOT) >> 4),
                                        da0 + (((unsigned)((zi + 2) & (kTczRing - 1)) * SLOT) >> 4)};
#pragma unroll 1
                for (int c = 0; c < a.nch; ++c) {
                    const uint64_t ca = (uint64_t)((2u * c * kTczSlabPitch) >> 4);
                    const uint64_t cb = db0 + (uint64_t)((c * 27u * 32u * NB) >> 4);
#pragma unroll
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;
                        const uint64_t da = sa[dz] + ca + (uint64_t)(((dy * kTcHX + dx) * 16) >> 4);
                        const uint64_t db = cb + (uint64_t)((tap * 32 * NB) >> 4);
                        mma_tf32(acc, da, db, idesc, (c > 0 || tap > 0) ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&mdone[zi & 1]))
                             : "memory");
                // the slot of plane zi-1 is free once output zi-1's MMAs are done: plane zi+3 goes there
                if (zi >= 1 && zi + 3 < np) {
                    ok = wait(&mdone[(zi - 1) & 1], ((zi - 1) >> 1) & 1);
                    if (ok) load_plane(zi + 3);
                }
            }
            // every MMA issued, then every load issued, must finish before the
            // shared memory and TMEM are given up
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&fin))
                         : "memory");
            const int saved = abort_flag;
            abort_flag = 0;  // the drain below must not stop early
            bool drained = wait(&fin, 0);
            if (!w_seen) drained = wait(&wbar, 0) && drained;
            for (int sl = 0; sl < kTczRing; ++sl)
                if (last_q[sl] > seen_q[sl]) drained = wait(&pfull[sl], (last_q[sl] >> 2) & 1) && drained;
            if (!ok || !drained || saved) {
                abort_flag = 1;
                atomicExch(a.err, 1);
            }
        }
    } else {
        const unsigned row = tmem + ((unsigned)(32 * warp) << 16);
        const int m = 32 * warp + lane;
        const int x = x0 + (m & 7), y = y0 + (m >> 3);
        const bool inside = x < a.X && y < a.Y;
        float bv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) bv[j] = (a.bias && j < a.cout) ? a.bias[j] : 0.f;
        for (int zi = 0; zi < nz; ++zi) {
            bool ok = false;
            for (unsigned it = 0; it < kTcSpinW; ++it) {
                if (mbar_try_wait(&mdone[zi & 1], (zi >> 1) & 1)) {
                    ok = true;
                    break;
                }
                if (abort_flag) break;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v[NB];
#pragma unroll
            for (int c = 0; c < NB; c += 16) tmem_ld16(row + (unsigned)((zi & 1) * NB + c), v + c);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive1(&afree[zi & 1]);
            if (inside) {
                const long long node = (long long)((z0 + zi) * a.Y + y) * a.X + x;
                float* o = a.out + b * a.out_bs + node * a.out_pitch;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j >= a.cout) break;
                    float val = v[j] + bv[j];
                    if (a.mode == 1) val = val > 0.f ? val : kSlope * val;
                    o[j] = val;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

// Weight image of one stride-1 layer for k_conv_tc.  Forward (flip = 0): the
// GEMM's output channel is the layer's co and its K channel the layer's ci;
// backward data (flip = 1): output channel = ci, K channel = co, tap mirrored.
// img[nblk][nch][tap][kh][ng][r][q] = W[co][tap'][ci] with the GEMM output
// channel nblk NB + 8 ng + r and K channel 8 c + 4 kh + q (0 outside).
__global__ void k_tc_image(const float* __restrict__ W, int cin, int coutp, int flip, int NB, int nblk, int nch,
                           float* __restrict__ img) {
    const long long n = (long long)nblk * nch * 27 * NB * 8;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long r = i;
    const int q = (int)(r % 4);
    r /= 4;
    const int rr = (int)(r % 8);
    r /= 8;
    const int ng = (int)(r % (NB / 8));
    r /= NB / 8;
    const int kh = (int)(r % 2);
    r /= 2;
    const int tap = (int)(r % 27);
    r /= 27;
    const int c = (int)(r % nch);
    const int blk = (int)(r / nch);
    const int gout = blk * NB + 8 * ng + rr;  // GEMM output channel
    const int gk = 8 * c + 4 * kh + q;        // GEMM K channel
    float v = 0.f;
    if (!flip) {
        if (gout < coutp && gk < cin) v = W[((long long)gout * 27 + tap) * cin + gk];
    } else {
        if (gout < cin && gk < coutp) v = W[((long long)gk * 27 + (26 - tap)) * cin + gout];
    }
    img[i] = v;
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

struct Work {
    int nx, ny, nz, B;
    int X[4], Y[4], Z[4];
    long long N[4];
    // activations
    float *a0 = nullptr, *cat0 = nullptr, *b1 = nullptr, *cat1 = nullptr, *b2 = nullptr, *cat2 = nullptr,
          *b3 = nullptr, *c3 = nullptr, *y2 = nullptr, *y1 = nullptr, *y0 = nullptr;
    // training
    bool train = false;
    float *x0 = nullptr, *t = nullptr, *g = nullptr;
    float *gg = nullptr, *g_y0 = nullptr, *g_cat0 = nullptr, *g_y1 = nullptr, *g_cat1 = nullptr, *g_y2 = nullptr,
          *g_cat2 = nullptr, *g_c3 = nullptr, *g_b3 = nullptr, *g_b2 = nullptr, *g_b1 = nullptr, *g_a0 = nullptr;
    float* part = nullptr;
    long long part_cap = 0;
    float* split = nullptr;  // input-channel split partials of the stride-2 layers
    long long split_cap = 0;
    double* red = nullptr;   // reduction partials (2 * kRedBlocks)
    double* sc = nullptr;    // [0] = loss DOF count, [1] = energy-loss gradient scale
    cudaGraphExec_t exec = nullptr;         // train step, mean squared error
    unsigned long long graph_kernels = 0;  // kernels one replay of exec runs
    // energy loss: per-sample moduli and masks staged from the operators,
    // masked output / target, their images under K, per-sample dot partials
    // and gradient coefficients
    bool energy = false;
    float *Es = nullptr, *gm = nullptr, *tm = nullptr, *Kg = nullptr, *Kt = nullptr;
    double *epart = nullptr, *coef = nullptr;
    uint8_t* ms = nullptr;
    int* kerr = nullptr;
    gmg::GSym gs{};
    cudaGraphExec_t exec_energy = nullptr;
    unsigned long long graph_kernels_energy = 0;
    std::vector<void*> allocs;
};

}  // namespace

struct gmg_net {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    LayerTable T{};
    long long n_int = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr, *Wr = nullptr, *Wf = nullptr, *Wb = nullptr;
    double* adam = nullptr;  // t, c1, c2
    float* lr = nullptr;
    float* loss = nullptr;
    std::vector<Work*> works;
    std::vector<void*> allocs;
    // tensor-core (TF32) stride-1 convolutions: per layer and direction
    // (0 forward, 1 backward data) the weight image and its GEMM blocking
    int arith = GMG_NET_FP32;
    bool tcz = true;  // z-marching tensor-core kernel where a layer fits it (else one tile per CTA)
    float* img[kLayers][2] = {};
    int img_nb[kLayers][2] = {}, img_nblk[kLayers][2] = {}, img_nch[kLayers][2] = {};
    int* kerr = nullptr;  // sticky error word of the tensor-core kernels
    // warm start scratch
    float *ws_g = nullptr, *ws_kg = nullptr, *ws_x = nullptr;
    long long ws_cap = 0;
    double *ws_red = nullptr, *ws_alpha = nullptr;
};

namespace {

template <class T>
int dalloc(std::vector<void*>& owner, T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GMG_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    owner.push_back(q);
    *p = static_cast<T*>(q);
    return GMG_OK;
}

void free_all(std::vector<void*>& v) {
    for (void* p : v) cudaFree(p);
    v.clear();
}

// API parameter offsets (out layer with 3 output channels)
long long api_offset(int l) {
    long long k = 0;
    for (int i = 0; i < l; ++i) k += (long long)kDefs[i].cout * 27 * kDefs[i].cin + kDefs[i].cout;
    return k;
}

LayerTable make_table(long long* total) {
    LayerTable T{};
    long long k = 0;
    for (int l = 0; l < kLayers; ++l) {
        T.cin[l] = kDefs[l].cin;
        T.coutp[l] = cpad4(kDefs[l].cout);
        T.woff[l] = k;
        k += (long long)T.coutp[l] * 27 * T.cin[l];
        T.boff[l] = k;
        k += T.coutp[l];
    }
    *total = k;
    return T;
}

// ---- tensor-core convolution (stride 1)

template <int NB>
int tcz_attr() {
    CU(cudaFuncSetAttribute(k_conv_tcz<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024 + 1024));
    return GMG_OK;
}

int tc_nb(int cout) { return cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16); }

template <int NB>
int tc_attr() {
    CU(cudaFuncSetAttribute(k_conv_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcGeom<NB>::SMEM));
    return GMG_OK;
}

// Allocates the forward weight image of every stride-1 layer with its GEMM
// blocking.  (k_tc_image also lays out the backward-data form, flip = 1; the
// backward passes stay on the FP32 path: TF32 gradients lose ~8 % relative
// accuracy on the first layer after eleven layers of cancellation.)
int alloc_images(gmg_net* net) {
    TRY(tc_attr<16>());
    TRY(tc_attr<32>());
    TRY(tc_attr<64>());
    TRY(tcz_attr<16>());
    TRY(tcz_attr<32>());
    TRY(tcz_attr<64>());
    for (int l = 0; l < kLayers; ++l) {
        if (kDefs[l].stride != 1) continue;
        for (int dir = 0; dir < 1; ++dir) {
            const int gout = dir == 0 ? net->T.coutp[l] : kDefs[l].cin;  // GEMM output channels
            const int gk = dir == 0 ? kDefs[l].cin : net->T.coutp[l];    // GEMM K channels
            const int nb = tc_nb(gout);
            net->img_nb[l][dir] = nb;
            net->img_nblk[l][dir] = (gout + nb - 1) / nb;
            net->img_nch[l][dir] = (gk + 7) / 8;
            const long long n = (long long)net->img_nblk[l][dir] * net->img_nch[l][dir] * 27 * nb * 8;
            TRY(dalloc(net->allocs, &net->img[l][dir], n));
        }
    }
    return GMG_OK;
}

// Rebuilds every weight image from the rounded weights Wr.
int build_images(gmg_net* net, cudaStream_t s) {
    for (int l = 0; l < kLayers; ++l)
        for (int dir = 0; dir < 2; ++dir) {
            if (!net->img[l][dir]) continue;
            const int nb = net->img_nb[l][dir], nblk = net->img_nblk[l][dir], nch = net->img_nch[l][dir];
            const long long n = (long long)nblk * nch * 27 * nb * 8;
            k_tc_image<<<blocks_for(n, 256), 256, 0, s>>>(net->Wr + net->T.woff[l], kDefs[l].cin, net->T.coutp[l], dir,
                                                          nb, nblk, nch, net->img[l][dir]);
            note_launch();
        }
    return GMG_OK;
}

// Launches k_conv_tc for layer l in direction dir; returns 1 (nothing
// launched) when the input cannot be described by a tensor map.
int launch_conv_tc(gmg_net* net, int l, int dir, const float* in, int in_pitch, int cin, long long in_bs, int X, int Y,
                   int Z, int B, float* out, int out_pitch, int cout, long long out_bs, const float* bias,
                   const float* ref, int ref_pitch, long long ref_bs, int mode, int accumulate, cudaStream_t s) {
    CUtensorMap tm;
    const unsigned long long dims[5] = {(unsigned long long)cin, (unsigned long long)X, (unsigned long long)Y,
                                        (unsigned long long)Z, (unsigned long long)B};
    const unsigned long long st[4] = {4ULL * in_pitch, 4ULL * in_pitch * X, 4ULL * in_pitch * X * Y,
                                      4ULL * (unsigned long long)in_bs};
    const unsigned box[5] = {4, kTcHX, kTcHY, kTcHZ, 1};
    if (!gmg::encode_f32_map_strided(&tm, in, 5, dims, st, box)) return 1;
    TcConvArgs a{};
    a.out = out;
    a.out_pitch = out_pitch;
    a.cout = cout;
    a.img = net->img[l][dir];
    a.bias = bias;
    a.ref = ref;
    a.ref_pitch = ref_pitch;
    a.mode = mode;
    a.accumulate = accumulate;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.nch = net->img_nch[l][dir];
    a.out_bs = out_bs;
    a.ref_bs = ref_bs;
    a.err = net->kerr;
    const int nb = net->img_nb[l][dir];
    dim3 grid((unsigned)(((X + 7) / 8) * ((Y + 15) / 16) * Z), (unsigned)net->img_nblk[l][dir], (unsigned)B);
    switch (nb) {
        case 16: k_conv_tc<16><<<grid, 128, TcGeom<16>::SMEM, s>>>(tm, a); break;
        case 32: k_conv_tc<32><<<grid, 128, TcGeom<32>::SMEM, s>>>(tm, a); break;
        default: k_conv_tc<64><<<grid, 128, TcGeom<64>::SMEM, s>>>(tm, a); break;
    }
    note_launch();
    return GMG_OK;
}

// Shared memory of k_conv_tcz for a layer (weights + four plane slots), or 0
// when fewer than two CTAs would fit an SM: with a single CTA per SM the ring's
// one plane of prefetch leaves the loads exposed, and the one-tile-per-CTA
// kernel is faster (measured at 80^3: layer u0 307 us vs 189 us, while the
// 16-channel layers take 81-86 us vs 94-97 us).
size_t tcz_smem(int nb, int nch) {
    const size_t wb = (size_t)nch * 27 * 32 * nb;
    const size_t slot = (size_t)2 * nch * kTczSlabPitch;
    const size_t total = wb + kTczRing * slot + 1024;
    return total <= 113 * 1024 ? total : 0;
}

// Launches k_conv_tcz for the forward pass of stride-1 layer l; returns 1
// (nothing launched) when the layer does not suit it.
int launch_conv_tcz(gmg_net* net, int l, const float* in, int in_pitch, int cin, long long in_bs, int X, int Y, int Z,
                    int B, float* out, int out_pitch, int cout, long long out_bs, const float* bias, int mode,
                    cudaStream_t s) {
    if (net->img_nblk[l][0] != 1) return 1;
    const int nb = net->img_nb[l][0], nch = net->img_nch[l][0];
    const size_t smem = tcz_smem(nb, nch);
    if (!smem) return 1;
    CUtensorMap tm;
    const unsigned long long dims[5] = {(unsigned long long)cin, (unsigned long long)X, (unsigned long long)Y,
                                        (unsigned long long)Z, (unsigned long long)B};
    const unsigned long long st[4] = {4ULL * in_pitch, 4ULL * in_pitch * X, 4ULL * in_pitch * X * Y,
                                      4ULL * (unsigned long long)in_bs};
    const unsigned box[5] = {4, kTcHX, kTcHY, 1, 1};
    if (!gmg::encode_f32_map_strided(&tm, in, 5, dims, st, box)) return 1;
    const int tiles = ((X + 7) / 8) * ((Y + 15) / 16);
    const int per_sm = std::max(1, (int)(228 * 1024 / smem));
    int nzr = std::max(1, std::min(Z, (2 * 148 * per_sm + tiles * B - 1) / (tiles * B)));
    const int zr = (Z + nzr - 1) / nzr;
    nzr = (Z + zr - 1) / zr;
    TczArgs a{};
    a.out = out;
    a.out_pitch = out_pitch;
    a.cout = cout;
    a.img = net->img[l][0];
    a.bias = bias;
    a.mode = mode;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.nch = nch;
    a.nslab = 2 * nch;
    a.zr = zr;
    a.out_bs = out_bs;
    a.err = net->kerr;
    dim3 grid((unsigned)tiles, (unsigned)nzr, (unsigned)B);
    switch (nb) {
        case 16: k_conv_tcz<16><<<grid, 160, smem, s>>>(tm, a); break;
        case 32: k_conv_tcz<32><<<grid, 160, smem, s>>>(tm, a); break;
        default: k_conv_tcz<64><<<grid, 160, smem, s>>>(tm, a); break;
    }
    note_launch();
    return GMG_OK;
}

// ---- convolution launchers

template <int COB, int TY, int TZ, int S>
int conv_attr() {
    CU(cudaFuncSetAttribute(k_conv<COB, TY, TZ, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)ConvGeom<COB, TY, TZ, S>::SMEM));
    return GMG_OK;
}

// Opt-in shared-memory sizes of every k_conv instantiation (set before any
// launch or capture).
int conv_attrs() {
    TRY((conv_attr<64, 4, 4, 1>()));
    TRY((conv_attr<32, 8, 4, 1>()));
    TRY((conv_attr<16, 8, 8, 1>()));
    TRY((conv_attr<4, 16, 8, 1>()));
    TRY((conv_attr<64, 4, 4, 2>()));
    TRY((conv_attr<32, 8, 4, 2>()));
    TRY((conv_attr<16, 8, 8, 2>()));
    return GMG_OK;
}

template <int COB, int TY, int TZ, int S>
int launch_conv_t(const ConvArgs& a, int B, cudaStream_t s) {
    using Gm = ConvGeom<COB, TY, TZ, S>;
    const unsigned tiles = (unsigned)(((a.Xo + 7) / 8) * ((a.Yo + TY - 1) / TY) * ((a.Zo + TZ - 1) / TZ));
    const int splits = a.split_bs ? a.cin / a.ci_hi : 1;
    dim3 grid(tiles, (unsigned)((a.cout + COB - 1) / COB), (unsigned)(B * splits));
    k_conv<COB, TY, TZ, S><<<grid, Gm::NT, Gm::SMEM, s>>>(a);
    note_launch();
    return GMG_OK;
}

int launch_conv(ConvArgs a, int S, int B, cudaStream_t s) {
    if (a.cin % 4 || a.in_pitch % 4 || a.w_co % 4 || (reinterpret_cast<uintptr_t>(a.in) & 15) ||
        (reinterpret_cast<uintptr_t>(a.W) & 15))
        return fail(GMG_ERR_ARG, "conv: channel counts, pitches and pointers must be 16-byte aligned");
    if (a.ci_hi <= 0) a.ci_hi = a.cin;
    if (a.cin % a.ci_hi || a.ci_hi % 4) return fail(GMG_ERR_ARG, "conv: split must divide the input channels");
    const int c = a.cout;
    if (S == 1) {
        if (c % 64 == 0) return launch_conv_t<64, 4, 4, 1>(a, B, s);
        if (c % 32 == 0) return launch_conv_t<32, 8, 4, 1>(a, B, s);
        if (c % 16 == 0) return launch_conv_t<16, 8, 8, 1>(a, B, s);
        return launch_conv_t<4, 16, 8, 1>(a, B, s);
    }
    if (c % 64 == 0) return launch_conv_t<64, 4, 4, 2>(a, B, s);
    if (c % 32 == 0) return launch_conv_t<32, 8, 4, 2>(a, B, s);
    return launch_conv_t<16, 8, 8, 2>(a, B, s);
}

// out (cout channels) = act(conv(in) + bias) for layer l
int conv_fwd(gmg_net* net, int l, const float* in, int in_pitch, long long in_bs, int X, int Y, int Z, float* out,
             int out_pitch, int cout, long long out_bs, int B, cudaStream_t s, float* split = nullptr,
             long long split_cap = 0) {
    const LayerDef& d = kDefs[l];
    ConvArgs a{};
    a.in = in;
    a.in_pitch = in_pitch;
    a.cin = d.cin;
    a.out = out;
    a.out_pitch = out_pitch;
    a.cout = cout;
    a.W = net->Wf + net->T.woff[l];
    a.w_co = net->T.coutp[l];
    a.bias = net->Wr + net->T.boff[l];
    a.mode = d.act ? 1 : 0;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.Xo = d.stride == 1 ? X : (X - 1) / 2 + 1;
    a.Yo = d.stride == 1 ? Y : (Y - 1) / 2 + 1;
    a.Zo = d.stride == 1 ? Z : (Z - 1) / 2 + 1;
    a.in_bs = in_bs;
    a.out_bs = out_bs;
    if (net->arith == GMG_NET_TF32 && d.stride == 1) {
        int rc = net->tcz ? launch_conv_tcz(net, l, in, in_pitch, d.cin, in_bs, X, Y, Z, B, out, out_pitch, cout, out_bs,
                                            a.bias, a.mode, s)
                          : 1;
        if (rc == 1)
            rc = launch_conv_tc(net, l, 0, in, in_pitch, d.cin, in_bs, X, Y, Z, B, out, out_pitch, cout, out_bs, a.bias,
                                nullptr, 0, 0, a.mode, 0, s);
        if (rc != 1) return rc;
    }
    if (d.stride == 2 && split) {
        // few output tiles (coarse levels): split the input channels over more
        // blocks, then add the splits in order with bias and activation
        const int cob = cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16);
        const int ty = cob == 64 ? 4 : 8, tz = cob == 16 ? 8 : 4;
        const long long blocks = (long long)((a.Xo + 7) / 8) * ((a.Yo + ty - 1) / ty) * ((a.Zo + tz - 1) / tz) *
                                 ((cout + cob - 1) / cob) * B;
        int splits = 1;
        while (splits * 2 <= d.cin / 4 && blocks * splits < 2 * 148 && d.cin % (splits * 2 * 4) == 0) splits *= 2;
        const long long no = (long long)a.Xo * a.Yo * a.Zo;
        if (splits > 1 && (long long)splits * no * B * cout <= split_cap) {
            ConvArgs p = a;
            p.out = split;
            p.out_pitch = cout;
            p.out_bs = no * cout;
            p.split_bs = no * B * cout;
            p.ci_hi = d.cin / splits;
            p.bias = nullptr;
            p.mode = 0;
            TRY(launch_conv(p, 2, B, s));
            const long long n = no * B * cout;
            k_split_sum<<<blocks_for(n, 256), 256, 0, s>>>(split, splits, p.split_bs, no * B, cout, a.bias, d.act, out,
                                                           out_pitch, out_bs, no);
            note_launch();
            return GMG_OK;
        }
    }
    return launch_conv(a, d.stride, B, s);
}

// Backward data pass of stride-1 layer l: gin (cin channels) [+]= conv^T(gout),
// times lrelu'(ref) when ref is given.
int conv_bwd_s1(gmg_net* net, int l, const float* gout, int go_pitch, long long go_bs, float* gin, int gi_pitch,
                long long gi_bs, const float* ref, int ref_pitch, long long ref_bs, int accumulate, int X, int Y, int Z,
                int B, cudaStream_t s) {
    const LayerDef& d = kDefs[l];
    ConvArgs a{};
    a.in = gout;
    a.in_pitch = go_pitch;
    a.cin = net->T.coutp[l];
    a.out = gin;
    a.out_pitch = gi_pitch;
    a.cout = d.cin;
    a.W = net->Wb + net->T.woff[l];
    a.w_co = d.cin;
    a.bias = nullptr;
    a.ref = ref;
    a.ref_pitch = ref_pitch;
    a.mode = ref ? 2 : 0;
    a.accumulate = accumulate;
    a.X = a.Xo = X;
    a.Y = a.Yo = Y;
    a.Z = a.Zo = Z;
    a.in_bs = go_bs;
    a.out_bs = gi_bs;
    a.ref_bs = ref_bs;
    return launch_conv(a, 1, B, s);
}

// Backward data pass of stride-2 layer l (fine grid X, Y, Z): accumulate into gin, times lrelu'(ref).
int conv_bwd_s2(gmg_net* net, int l, const float* gout, int go_pitch, long long go_bs, float* gin, int gi_pitch,
                long long gi_bs, const float* ref, int ref_pitch, long long ref_bs, int X, int Y, int Z, int B,
                cudaStream_t s) {
    const LayerDef& d = kDefs[l];
    S2tArgs a{};
    a.go = gout;
    a.go_pitch = go_pitch;
    a.cout = net->T.coutp[l];
    a.W = net->Wr + net->T.woff[l];
    a.cin = d.cin;
    a.out = gin;
    a.out_pitch = gi_pitch;
    a.ref = ref;
    a.ref_pitch = ref_pitch;
    a.accumulate = 1;
    a.mode = ref ? 2 : 0;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.Xo = (X - 1) / 2 + 1;
    a.Yo = (Y - 1) / 2 + 1;
    a.Zo = (Z - 1) / 2 + 1;
    a.go_bs = go_bs;
    a.out_bs = gi_bs;
    a.ref_bs = ref_bs;
    const int cig = d.cin / 4;
    const int rows = 256 / cig;
    const int TY = rows >= 32 ? 8 : 4, TZ = rows / TY;
    dim3 grid((unsigned)(((X + 7) / 8) * ((Y + TY - 1) / TY) * ((Z + TZ - 1) / TZ)), 1, (unsigned)B);
    switch (cig) {
        case 4: k_conv_s2t<4><<<grid, 256, 0, s>>>(a); break;
        case 8: k_conv_s2t<8><<<grid, 256, 0, s>>>(a); break;
        case 16: k_conv_s2t<16><<<grid, 256, 0, s>>>(a); break;
        default: return fail(GMG_ERR_ARG, "conv_bwd_s2: unsupported channel count");
    }
    note_launch();
    return GMG_OK;
}

// Splits of the output nodes for the weight gradient of a layer.
// Blocks of k_wgrad resident on the whole GPU (the occupancy of the heavier
// instantiation times the SM count), so that the split grid fills whole waves.
long long wgrad_wave() {
    static long long n = 0;
    if (n == 0) {
        int dev = 0, sms = 0, r1 = 0, r2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r1, k_wgrad<1>, 256, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r2, k_wgrad<2>, 256, 0) != cudaSuccess)
            r1 = r2 = 2, (void)cudaGetLastError();
        n = (long long)sms * std::max(1, std::min(r1, r2));
    }
    return n;
}

int wgrad_splits(long long out_nodes, int task_blocks) {
    const long long target_blocks = wgrad_wave();
    long long sp = std::max<long long>(1, target_blocks / std::max(1, task_blocks));
    sp = std::min<long long>(sp, std::max<long long>(1, out_nodes / 128));
    return (int)std::min<long long>(sp, 4096);
}

long long wgrad_part_size(int l, long long out_nodes) {
    const int coutp = cpad4(kDefs[l].cout), cin = kDefs[l].cin;
    const int tasks = (coutp / 4) * (cin / 4) * 9;
    const int tb = (tasks + 255) / 256;
    const long long per = (long long)coutp * 27 * cin + coutp;
    return (long long)wgrad_splits(out_nodes, tb) * per;
}

// G slice of layer l = gradient from (in, gout) over the batch
int wgrad(gmg_net* net, Work* w, int l, const float* in, int in_pitch, long long in_bs, int X, int Y, int Z,
          const float* gout, int go_pitch, long long go_bs, cudaStream_t s) {
    const LayerDef& d = kDefs[l];
    WgArgs a{};
    a.in = in;
    a.in_pitch = in_pitch;
    a.cin = d.cin;
    a.go = gout;
    a.go_pitch = go_pitch;
    a.coutp = net->T.coutp[l];
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.Xo = d.stride == 1 ? X : (X - 1) / 2 + 1;
    a.Yo = d.stride == 1 ? Y : (Y - 1) / 2 + 1;
    a.Zo = d.stride == 1 ? Z : (Z - 1) / 2 + 1;
    a.B = w->B;
    a.in_bs = in_bs;
    a.go_bs = go_bs;
    const long long out_nodes = (long long)a.Xo * a.Yo * a.Zo * w->B;
    const int tasks = (a.coutp / 4) * (a.cin / 4) * 9;
    const int tb = (tasks + 255) / 256;
    const int splits = wgrad_splits(out_nodes, tb);
    a.nodes_per_split = (out_nodes + splits - 1) / splits;
    const long long per = (long long)a.coutp * 27 * a.cin + a.coutp;
    a.part = w->part;
    a.part_stride = per;
    if ((long long)splits * per > w->part_cap) return fail(GMG_ERR_ARG, "wgrad: partial buffer too small");
    dim3 grid((unsigned)splits, (unsigned)tb);
    if (d.stride == 1) k_wgrad<1><<<grid, 256, 0, s>>>(a);
    else k_wgrad<2><<<grid, 256, 0, s>>>(a);
    k_sum_splits<<<blocks_for(per, 256), 256, 0, s>>>(w->part, per, splits, per, net->G + net->T.woff[l]);
    note_launch(2);
    return GMG_OK;
}

int upsample(const float* in, int pi, long long in_bs, float* out, int po, long long out_bs, int C, int Xc, int Yc,
             int Zc, int B, cudaStream_t s) {
    const long long n = (long long)(2 * Xc - 1) * (2 * Yc - 1) * (2 * Zc - 1) * (C / 4) * B;
    k_upsample<<<blocks_for(n, 256), 256, 0, s>>>(in, pi, out, po, C, Xc, Yc, Zc, in_bs, out_bs, B);
    note_launch();
    return GMG_OK;
}

int upsample_adj(const float* g, int pg, long long g_bs, float* out, int po, long long out_bs, const float* ref, int pr,
                 long long ref_bs, int C, int Xc, int Yc, int Zc, int B, cudaStream_t s) {
    const long long n = (long long)Xc * Yc * Zc * (C / 4) * B;
    k_upsample_adj<<<blocks_for(n, 256), 256, 0, s>>>(g, pg, out, po, ref, pr, C, Xc, Yc, Zc, g_bs, out_bs, ref_bs, B);
    note_launch();
    return GMG_OK;
}

// ---- workspaces

int check_dims(int nx, int ny, int nz, int B) {
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8 || B < 1)
        return fail(GMG_ERR_ARG, "warm-start network: nx, ny, nz must be multiples of 8 (>= 8) and batch >= 1");
    return GMG_OK;
}

int get_work(gmg_net* net, int nx, int ny, int nz, int B, bool train, Work** out) {
    for (Work* w : net->works)
        if (w->nx == nx && w->ny == ny && w->nz == nz && w->B == B && (w->train || !train)) {
            *out = w;
            return GMG_OK;
        }
    Work* w = new Work();
    w->nx = nx;
    w->ny = ny;
    w->nz = nz;
    w->B = B;
    w->train = train;
    for (int l = 0; l < 4; ++l) {
        w->X[l] = (nx >> l) + 1;
        w->Y[l] = (ny >> l) + 1;
        w->Z[l] = (nz >> l) + 1;
        w->N[l] = (long long)w->X[l] * w->Y[l] * w->Z[l];
    }
    auto al = [&](float** p, long long per_node, int lev) { return dalloc(w->allocs, p, (size_t)(per_node * w->N[lev] * B)); };
    int rc = GMG_OK;
    auto chain = [&](int r) { if (rc == GMG_OK) rc = r; };
    chain(al(&w->a0, 16, 0));
    chain(al(&w->cat0, 48, 0));
    chain(al(&w->b1, 32, 1));
    chain(al(&w->cat1, 96, 1));
    chain(al(&w->b2, 64, 2));
    chain(al(&w->cat2, 128, 2));
    chain(al(&w->b3, 64, 3));
    chain(al(&w->c3, 64, 3));
    chain(al(&w->y2, 64, 2));
    chain(al(&w->y1, 32, 1));
    chain(al(&w->y0, 16, 0));
    chain(al(&w->g, 4, 0));
    chain(dalloc(w->allocs, &w->red, 2 * kRedBlocks));
    // split partials: at most 16 splits of the level-1..3 outputs of one stride-2 layer
    w->split_cap = 16LL * w->N[1] * 32 * B;
    chain(dalloc(w->allocs, &w->split, (size_t)w->split_cap));
    chain(dalloc(w->allocs, &w->sc, 4));
    if (train) {
        chain(al(&w->x0, GMG_NET_IN, 0));
        chain(al(&w->t, 3, 0));
        chain(al(&w->gg, 4, 0));
        chain(al(&w->g_y0, 16, 0));
        chain(al(&w->g_cat0, 48, 0));
        chain(al(&w->g_y1, 32, 1));
        chain(al(&w->g_cat1, 96, 1));
        chain(al(&w->g_y2, 64, 2));
        chain(al(&w->g_cat2, 128, 2));
        chain(al(&w->g_c3, 64, 3));
        chain(al(&w->g_b3, 64, 3));
        chain(al(&w->g_b2, 64, 2));
        chain(al(&w->g_b1, 32, 1));
        chain(al(&w->g_a0, 16, 0));
        long long cap = 0;
        for (int l = 0; l < kLayers; ++l) {
            const int lev_out = l <= L_E0B ? 0 : l <= L_E1 ? 1 : l <= L_E2 ? 2 : l <= L_E3 ? 3 : l == L_U2 ? 2 : l == L_U1 ? 1 : 0;
            cap = std::max(cap, wgrad_part_size(l, w->N[lev_out] * B));
        }
        w->part_cap = cap;
        chain(dalloc(w->allocs, &w->part, (size_t)cap));
    }
    if (rc != GMG_OK) {
        free_all(w->allocs);
        delete w;
        return rc;
    }
    net->works.push_back(w);
    *out = w;
    return GMG_OK;
}

int ensure_energy(Work* w) {
    if (w->energy) return GMG_OK;
    const long long n3 = 3 * w->N[0] * w->B;
    const long long ne = (long long)w->nx * w->ny * w->nz * w->B;
    TRY(dalloc(w->allocs, &w->Es, ne));
    TRY(dalloc(w->allocs, &w->gm, n3));
    TRY(dalloc(w->allocs, &w->tm, n3));
    TRY(dalloc(w->allocs, &w->Kg, n3));
    TRY(dalloc(w->allocs, &w->Kt, n3));
    TRY(dalloc(w->allocs, &w->epart, 3LL * kEnergyBlocks * w->B));
    TRY(dalloc(w->allocs, &w->coef, 2LL * w->B));
    TRY(dalloc(w->allocs, &w->ms, w->N[0] * w->B));
    TRY(dalloc(w->allocs, &w->kerr, 4));
    CU(cudaMemset(w->kerr, 0, sizeof(int) * 4));
    w->energy = true;
    return GMG_OK;
}

// Forward pass: x (pitch 8) -> g (pitch gp, gc channels written), activations kept in w.
int forward(gmg_net* net, Work* w, const float* x, float* g, int gp, int gc, cudaStream_t s) {
    const int B = w->B;
    const int* X = w->X;
    const int* Y = w->Y;
    const int* Z = w->Z;
    const long long* N = w->N;
    TRY(conv_fwd(net, L_E0A, x, GMG_NET_IN, GMG_NET_IN * N[0], X[0], Y[0], Z[0], w->a0, 16, 16, 16 * N[0], B, s));
    TRY(conv_fwd(net, L_E0B, w->a0, 16, 16 * N[0], X[0], Y[0], Z[0], w->cat0 + 32, 48, 16, 48 * N[0], B, s));
    TRY(conv_fwd(net, L_D1, w->cat0 + 32, 48, 48 * N[0], X[0], Y[0], Z[0], w->b1, 32, 32, 32 * N[1], B, s, w->split, w->split_cap));
    TRY(conv_fwd(net, L_E1, w->b1, 32, 32 * N[1], X[1], Y[1], Z[1], w->cat1 + 64, 96, 32, 96 * N[1], B, s));
    TRY(conv_fwd(net, L_D2, w->cat1 + 64, 96, 96 * N[1], X[1], Y[1], Z[1], w->b2, 64, 64, 64 * N[2], B, s, w->split, w->split_cap));
    TRY(conv_fwd(net, L_E2, w->b2, 64, 64 * N[2], X[2], Y[2], Z[2], w->cat2 + 64, 128, 64, 128 * N[2], B, s));
    TRY(conv_fwd(net, L_D3, w->cat2 + 64, 128, 128 * N[2], X[2], Y[2], Z[2], w->b3, 64, 64, 64 * N[3], B, s, w->split, w->split_cap));
    TRY(conv_fwd(net, L_E3, w->b3, 64, 64 * N[3], X[3], Y[3], Z[3], w->c3, 64, 64, 64 * N[3], B, s));
    TRY(upsample(w->c3, 64, 64 * N[3], w->cat2, 128, 128 * N[2], 64, X[3], Y[3], Z[3], B, s));
    TRY(conv_fwd(net, L_U2, w->cat2, 128, 128 * N[2], X[2], Y[2], Z[2], w->y2, 64, 64, 64 * N[2], B, s));
    TRY(upsample(w->y2, 64, 64 * N[2], w->cat1, 96, 96 * N[1], 64, X[2], Y[2], Z[2], B, s));
    TRY(conv_fwd(net, L_U1, w->cat1, 96, 96 * N[1], X[1], Y[1], Z[1], w->y1, 32, 32, 32 * N[1], B, s));
    TRY(upsample(w->y1, 32, 32 * N[1], w->cat0, 48, 48 * N[0], 32, X[1], Y[1], Z[1], B, s));
    TRY(conv_fwd(net, L_U0, w->cat0, 48, 48 * N[0], X[0], Y[0], Z[0], w->y0, 16, 16, 16 * N[0], B, s));
    TRY(conv_fwd(net, L_OUT, w->y0, 16, 16 * N[0], X[0], Y[0], Z[0], g, gp, gc, (long long)gp * N[0], B, s));
    return GMG_OK;
}

// Loss, backward pass and Adam update (training workspace, inputs staged in
// x0 / t, and for the energy loss the moduli / masks in Es / ms).
int train_kernels(gmg_net* net, Work* w, bool energy, cudaStream_t s) {
    const int B = w->B;
    const int* X = w->X;
    const int* Y = w->Y;
    const int* Z = w->Z;
    const long long* N = w->N;
    const long long nodes = N[0] * B;
    if (!energy) {
        k_count_free<<<kRedBlocks, kRedThreads, 0, s>>>(w->x0, nodes, w->red);
        k_finish_sum<<<1, 256, 0, s>>>(w->red, kRedBlocks, 3.0, w->sc, 0);
        note_launch(2);
    }
    TRY(forward(net, w, w->x0, w->g, 4, 4, s));
    if (!energy) {
        k_loss<<<kRedBlocks, kRedThreads, 0, s>>>(w->g, w->t, w->x0, nodes, w->sc, w->gg, w->red);
        k_loss_finish<<<1, 256, 0, s>>>(w->red, kRedBlocks, w->sc, net->loss);
        note_launch(2);
    } else {
        const long long n3 = 3 * N[0];
        const long long ne = (long long)w->nx * w->ny * w->nz;
        k_energy_prep<<<blocks_for(n3 * B, 256), 256, 0, s>>>(w->g, w->t, w->ms, N[0], B, w->gm, w->tm);
        note_launch();
        for (int b = 0; b < B; ++b) {
            gmg::FineArgs a{};
            a.nx = w->nx;
            a.ny = w->ny;
            a.nz = w->nz;
            a.E = w->Es + b * ne;
            a.mask = w->ms + b * N[0];
            a.err = w->kerr;
            a.xin = w->gm + b * n3;
            a.out = w->Kg + b * n3;
            gmg::launch_fine(gmg::FM_APPLY, 0, 0, a, w->gs, s);
            a.xin = w->tm + b * n3;
            a.out = w->Kt + b * n3;
            gmg::launch_fine(gmg::FM_APPLY, 0, 0, a, w->gs, s);
        }
        k_energy_dots<<<dim3(kEnergyBlocks, B), kRedThreads, 0, s>>>(w->gm, w->Kg, w->tm, w->Kt, n3, w->epart);
        k_energy_finish<<<1, 256, 0, s>>>(w->epart, kEnergyBlocks, B, w->coef, net->loss);
        k_energy_grad<<<blocks_for(nodes, 256), 256, 0, s>>>(w->Kg, w->Kt, N[0], B, w->coef, w->gg);
        note_launch(3);
    }
    // out
    TRY(wgrad(net, w, L_OUT, w->y0, 16, 16 * N[0], X[0], Y[0], Z[0], w->gg, 4, 4 * N[0], s));
    TRY(conv_bwd_s1(net, L_OUT, w->gg, 4, 4 * N[0], w->g_y0, 16, 16 * N[0], w->y0, 16, 16 * N[0], 0, X[0], Y[0], Z[0], B, s));
    // u0
    TRY(wgrad(net, w, L_U0, w->cat0, 48, 48 * N[0], X[0], Y[0], Z[0], w->g_y0, 16, 16 * N[0], s));
    TRY(conv_bwd_s1(net, L_U0, w->g_y0, 16, 16 * N[0], w->g_cat0, 48, 48 * N[0], nullptr, 0, 0, 0, X[0], Y[0], Z[0], B, s));
    TRY(upsample_adj(w->g_cat0, 48, 48 * N[0], w->g_y1, 32, 32 * N[1], w->y1, 32, 32 * N[1], 32, X[1], Y[1], Z[1], B, s));
    // u1
    TRY(wgrad(net, w, L_U1, w->cat1, 96, 96 * N[1], X[1], Y[1], Z[1], w->g_y1, 32, 32 * N[1], s));
    TRY(conv_bwd_s1(net, L_U1, w->g_y1, 32, 32 * N[1], w->g_cat1, 96, 96 * N[1], nullptr, 0, 0, 0, X[1], Y[1], Z[1], B, s));
    TRY(upsample_adj(w->g_cat1, 96, 96 * N[1], w->g_y2, 64, 64 * N[2], w->y2, 64, 64 * N[2], 64, X[2], Y[2], Z[2], B, s));
    // u2
    TRY(wgrad(net, w, L_U2, w->cat2, 128, 128 * N[2], X[2], Y[2], Z[2], w->g_y2, 64, 64 * N[2], s));
    TRY(conv_bwd_s1(net, L_U2, w->g_y2, 64, 64 * N[2], w->g_cat2, 128, 128 * N[2], nullptr, 0, 0, 0, X[2], Y[2], Z[2], B, s));
    TRY(upsample_adj(w->g_cat2, 128, 128 * N[2], w->g_c3, 64, 64 * N[3], w->c3, 64, 64 * N[3], 64, X[3], Y[3], Z[3], B, s));
    // e3
    TRY(wgrad(net, w, L_E3, w->b3, 64, 64 * N[3], X[3], Y[3], Z[3], w->g_c3, 64, 64 * N[3], s));
    TRY(conv_bwd_s1(net, L_E3, w->g_c3, 64, 64 * N[3], w->g_b3, 64, 64 * N[3], w->b3, 64, 64 * N[3], 0, X[3], Y[3], Z[3], B, s));
    // d3 (level 2 -> 3): its input is s2 = cat2[64:128]
    TRY(wgrad(net, w, L_D3, w->cat2 + 64, 128, 128 * N[2], X[2], Y[2], Z[2], w->g_b3, 64, 64 * N[3], s));
    TRY(conv_bwd_s2(net, L_D3, w->g_b3, 64, 64 * N[3], w->g_cat2 + 64, 128, 128 * N[2], w->cat2 + 64, 128, 128 * N[2],
                    X[2], Y[2], Z[2], B, s));
    // e2
    TRY(wgrad(net, w, L_E2, w->b2, 64, 64 * N[2], X[2], Y[2], Z[2], w->g_cat2 + 64, 128, 128 * N[2], s));
    TRY(conv_bwd_s1(net, L_E2, w->g_cat2 + 64, 128, 128 * N[2], w->g_b2, 64, 64 * N[2], w->b2, 64, 64 * N[2], 0, X[2], Y[2],
                    Z[2], B, s));
    // d2
    TRY(wgrad(net, w, L_D2, w->cat1 + 64, 96, 96 * N[1], X[1], Y[1], Z[1], w->g_b2, 64, 64 * N[2], s));
    TRY(conv_bwd_s2(net, L_D2, w->g_b2, 64, 64 * N[2], w->g_cat1 + 64, 96, 96 * N[1], w->cat1 + 64, 96, 96 * N[1], X[1],
                    Y[1], Z[1], B, s));
    // e1
    TRY(wgrad(net, w, L_E1, w->b1, 32, 32 * N[1], X[1], Y[1], Z[1], w->g_cat1 + 64, 96, 96 * N[1], s));
    TRY(conv_bwd_s1(net, L_E1, w->g_cat1 + 64, 96, 96 * N[1], w->g_b1, 32, 32 * N[1], w->b1, 32, 32 * N[1], 0, X[1], Y[1],
                    Z[1], B, s));
    // d1
    TRY(wgrad(net, w, L_D1, w->cat0 + 32, 48, 48 * N[0], X[0], Y[0], Z[0], w->g_b1, 32, 32 * N[1], s));
    TRY(conv_bwd_s2(net, L_D1, w->g_b1, 32, 32 * N[1], w->g_cat0 + 32, 48, 48 * N[0], w->cat0 + 32, 48, 48 * N[0], X[0],
                    Y[0], Z[0], B, s));
    // e0b
    TRY(wgrad(net, w, L_E0B, w->a0, 16, 16 * N[0], X[0], Y[0], Z[0], w->g_cat0 + 32, 48, 48 * N[0], s));
    TRY(conv_bwd_s1(net, L_E0B, w->g_cat0 + 32, 48, 48 * N[0], w->g_a0, 16, 16 * N[0], w->a0, 16, 16 * N[0], 0, X[0], Y[0],
                    Z[0], B, s));
    // e0a
    TRY(wgrad(net, w, L_E0A, w->x0, GMG_NET_IN, GMG_NET_IN * N[0], X[0], Y[0], Z[0], w->g_a0, 16, 16 * N[0], s));
    // Adam
    k_sumsq_f<<<kRedBlocks, kRedThreads, 0, s>>>(net->G, net->n_int, w->red);
    k_adam_tick<<<1, 256, 0, s>>>(net->adam, w->red, kRedBlocks, net->lr + 1);
    k_adam<<<blocks_for(net->n_int, 256), 256, 0, s>>>(net->T, net->n_int, net->P, net->M, net->V, net->G, net->Wr,
                                                       net->Wf, net->Wb, net->adam, net->lr);
    note_launch(3);
    if (net->arith == GMG_NET_TF32) TRY(build_images(net, s));
    return GMG_OK;
}

int round_all(gmg_net* net) {
    k_round_all<<<blocks_for(net->n_int, 256), 256, 0, net->stream>>>(net->T, net->n_int, net->P, net->Wr, net->Wf, net->Wb);
    note_launch();
    TRY(build_images(net, net->stream));
    CU(cudaGetLastError());
    return GMG_OK;
}

// Destroys the captured train-step graphs (they depend on the arithmetic).
void drop_graphs(gmg_net* net) {
    for (Work* w : net->works) {
        if (w->exec) cudaGraphExecDestroy(w->exec);
        if (w->exec_energy) cudaGraphExecDestroy(w->exec_energy);
        w->exec = w->exec_energy = nullptr;
    }
}

int api_to_internal(gmg_net* net, const float* params) {
    cudaStream_t s = net->stream;
    CU(cudaMemsetAsync(net->P, 0, sizeof(float) * net->n_int, s));
    const long long head = api_offset(L_OUT);  // layers 0..10 share the layout
    CU(cudaMemcpyAsync(net->P, params, sizeof(float) * head, cudaMemcpyDeviceToDevice, s));
    const long long nw = 3LL * 27 * 16;
    CU(cudaMemcpyAsync(net->P + net->T.woff[L_OUT], params + head, sizeof(float) * nw, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(net->P + net->T.boff[L_OUT], params + head + nw, sizeof(float) * 3, cudaMemcpyDeviceToDevice, s));
    return GMG_OK;
}

int internal_to_api(gmg_net* net, const float* src, float* params) {
    cudaStream_t s = net->stream;
    const long long head = api_offset(L_OUT);
    CU(cudaMemcpyAsync(params, src, sizeof(float) * head, cudaMemcpyDeviceToDevice, s));
    const long long nw = 3LL * 27 * 16;
    CU(cudaMemcpyAsync(params + head, src + net->T.woff[L_OUT], sizeof(float) * nw, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(params + head + nw, src + net->T.boff[L_OUT], sizeof(float) * 3, cudaMemcpyDeviceToDevice, s));
    return GMG_OK;
}

int reset_state(gmg_net* net) {
    cudaStream_t s = net->stream;
    CU(cudaMemsetAsync(net->M, 0, sizeof(float) * net->n_int, s));
    CU(cudaMemsetAsync(net->V, 0, sizeof(float) * net->n_int, s));
    CU(cudaMemsetAsync(net->G, 0, sizeof(float) * net->n_int, s));
    CU(cudaMemsetAsync(net->adam, 0, sizeof(double) * 4, s));
    return GMG_OK;
}

}  // namespace

extern "C" {

long long gmg_net_num_params(void) { return api_offset(kLayers); }

int gmg_net_layer_shape(int layer, int shape[4]) {
    if (layer < 0 || layer >= kLayers || !shape) return fail(GMG_ERR_ARG, "layer index out of range");
    shape[0] = kDefs[layer].cin;
    shape[1] = kDefs[layer].cout;
    shape[2] = kDefs[layer].stride;
    shape[3] = kDefs[layer].act;
    return GMG_OK;
}

int gmg_net_create(gmg_net** out, const float* params, void* stream) {
    if (!out || !params) return fail(GMG_ERR_ARG, "null argument");
    *out = nullptr;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    gmg_net* net = new gmg_net();
    net->stream = static_cast<cudaStream_t>(stream);
    net->T = make_table(&net->n_int);
    int rc = GMG_OK;
    auto chain = [&](int r) { if (rc == GMG_OK) rc = r; };
    chain(dalloc(net->allocs, &net->P, net->n_int));
    chain(dalloc(net->allocs, &net->M, net->n_int));
    chain(dalloc(net->allocs, &net->V, net->n_int));
    chain(dalloc(net->allocs, &net->G, net->n_int));
    chain(dalloc(net->allocs, &net->Wr, net->n_int));
    chain(dalloc(net->allocs, &net->Wf, net->n_int));
    chain(dalloc(net->allocs, &net->Wb, net->n_int));
    chain(dalloc(net->allocs, &net->adam, 4));
    chain(dalloc(net->allocs, &net->lr, 4));  // lr, clip
    chain(dalloc(net->allocs, &net->loss, 4));
    chain(dalloc(net->allocs, &net->ws_red, 4 * kRedBlocks));
    chain(dalloc(net->allocs, &net->kerr, 4));
    if (rc == GMG_OK) rc = alloc_images(net);
    if (rc == GMG_OK && cudaMemsetAsync(net->kerr, 0, 16, net->stream) != cudaSuccess) rc = GMG_ERR_CUDA;
    chain(dalloc(net->allocs, &net->ws_alpha, 8));
    if (rc == GMG_OK) rc = conv_attrs();
    if (rc == GMG_OK) rc = api_to_internal(net, params);
    if (rc == GMG_OK) rc = reset_state(net);
    if (rc == GMG_OK) rc = round_all(net);
    if (rc != GMG_OK) {
        free_all(net->allocs);
        delete net;
        return rc;
    }
    *out = net;
    return GMG_OK;
}

int gmg_net_set_params(gmg_net* net, const float* params) {
    if (!net || !params) return fail(GMG_ERR_ARG, "null argument");
    TRY(api_to_internal(net, params));
    TRY(reset_state(net));
    return round_all(net);
}

int gmg_net_get_params(gmg_net* net, float* params) {
    if (!net || !params) return fail(GMG_ERR_ARG, "null argument");
    return internal_to_api(net, net->P, params);
}

int gmg_net_get_grads(gmg_net* net, float* grads) {
    if (!net || !grads) return fail(GMG_ERR_ARG, "null argument");
    return internal_to_api(net, net->G, grads);
}

int gmg_net_set_arith(gmg_net* net, int arith) {
    if (!net || (arith != GMG_NET_FP32 && arith != GMG_NET_TF32)) return fail(GMG_ERR_ARG, "bad arithmetic mode");
    if (arith != net->arith) {
        CU(cudaStreamSynchronize(net->stream));
        drop_graphs(net);
        net->arith = arith;
        // the images follow the weights only while TF32 is selected: refresh
        // them from the current (possibly trained) weights
        if (arith == GMG_NET_TF32) {
            TRY(build_images(net, net->stream));
            CU(cudaGetLastError());
        }
    }
    return GMG_OK;
}

int gmg_net_status(gmg_net* net) {
    if (!net) return fail(GMG_ERR_ARG, "null argument");
    int e = 0;
    CU(cudaMemcpyAsync(&e, net->kerr, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
    CU(cudaStreamSynchronize(net->stream));
    if (e) return fail(GMG_ERR_CUDA, "a tensor-core convolution gave up waiting for its operands");
    return GMG_OK;
}

int gmg_net_forward(gmg_net* net, int nx, int ny, int nz, int batch, const float* x, float* g) {
    if (!net || !x || !g) return fail(GMG_ERR_ARG, "null argument");
    TRY(check_dims(nx, ny, nz, batch));
    Work* w = nullptr;
    TRY(get_work(net, nx, ny, nz, batch, false, &w));
    TRY(forward(net, w, x, g, 3, 3, net->stream));
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_net_train_step(gmg_net* net, int nx, int ny, int nz, int batch, const float* const* x, const float* const* t,
                       gmg_handle* const* ops, float lr, float clip, float* loss) {
    if (!net || !x || !t) return fail(GMG_ERR_ARG, "null argument");
    TRY(check_dims(nx, ny, nz, batch));
    for (int b = 0; b < batch; ++b)
        if (!x[b] || !t[b] || (ops && !ops[b])) return fail(GMG_ERR_ARG, "null sample pointer");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(GMG_ERR_ARG, "lr must be finite and >= 0");
    if (!std::isfinite(clip)) return fail(GMG_ERR_ARG, "clip must be finite");
    const bool energy = ops != nullptr;
    if (energy)
        for (int b = 0; b < batch; ++b) {
            const gmg::Level& l0 = ops[b]->lev[0];
            if (l0.nx != nx || l0.ny != ny || l0.nz != nz)
                return fail(GMG_ERR_ARG, "operator grid differs from the batch grid");
            if (std::memcmp(&ops[b]->gs, &ops[0]->gs, sizeof(gmg::GSym)) != 0)
                return fail(GMG_ERR_ARG, "the operators of one batch must share Poisson's ratio");
        }
    Work* w = nullptr;
    TRY(get_work(net, nx, ny, nz, batch, true, &w));
    if (energy) {
        TRY(ensure_energy(w));
        if (w->exec_energy && std::memcmp(&w->gs, &ops[0]->gs, sizeof(gmg::GSym)) != 0) {
            cudaGraphExecDestroy(w->exec_energy);
            w->exec_energy = nullptr;
        }
        w->gs = ops[0]->gs;
    }
    cudaStream_t s = net->stream;
    const long long N0 = w->N[0];
    const long long ne = (long long)nx * ny * nz;
    for (int b = 0; b < batch; ++b) {
        CU(cudaMemcpyAsync(w->x0 + b * GMG_NET_IN * N0, x[b], sizeof(float) * GMG_NET_IN * N0, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(w->t + b * 3 * N0, t[b], sizeof(float) * 3 * N0, cudaMemcpyDeviceToDevice, s));
        if (energy) {
            CU(cudaMemcpyAsync(w->Es + b * ne, ops[b]->E32, sizeof(float) * ne, cudaMemcpyDeviceToDevice, s));
            CU(cudaMemcpyAsync(w->ms + b * N0, ops[b]->lev[0].mask, N0, cudaMemcpyDeviceToDevice, s));
        }
    }
    const float hyper[2] = {lr, clip};
    CU(cudaMemcpyAsync(net->lr, hyper, sizeof(hyper), cudaMemcpyHostToDevice, s));
    cudaGraphExec_t& exec = energy ? w->exec_energy : w->exec;
    unsigned long long& kernels = energy ? w->graph_kernels_energy : w->graph_kernels;
    if (!exec) {
        if (!net->cap && cudaStreamCreateWithFlags(&net->cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return fail(GMG_ERR_CUDA, "cannot create the capture stream");
        }
        // captured kernels are counted when the graph runs, not here
        const unsigned long long before = gmg::g_kernel_launches.load();
        CU(cudaStreamBeginCapture(net->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = train_kernels(net, w, energy, net->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(net->cap, &graph);
        kernels = gmg::g_kernel_launches.load() - before;
        gmg::g_kernel_launches.fetch_sub(kernels);
        if (rc != GMG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ec != cudaSuccess) return fail(GMG_ERR_CUDA, std::string("train-step capture failed: ") + cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            exec = nullptr;
            return fail(GMG_ERR_CUDA, std::string("train-step graph instantiation failed: ") + cudaGetErrorString(ei));
        }
    }
    CU(cudaGraphLaunch(exec, s));
    note_launch(kernels);
    if (loss) CU(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_net_features(int nx, int ny, int nz, const float* rho, const double* f, const uint8_t* fixed, float* x,
                     void* stream) {
    if (!rho || !f || !fixed || !x) return fail(GMG_ERR_ARG, "null argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(GMG_ERR_ARG, "grid must be at least 1 x 1 x 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    double* red = nullptr;
    CU(cudaMallocAsync(&red, sizeof(double) * (4 * kRedBlocks + 4), s));
    k_load_stats<<<kRedBlocks, kRedThreads, 0, s>>>(f, nn, red);
    k_load_stats_finish<<<1, 256, 0, s>>>(red, kRedBlocks, red + 4 * kRedBlocks);
    k_features<<<blocks_for(nn, 256), 256, 0, s>>>(nx, ny, nz, rho, f, fixed, nullptr, red + 4 * kRedBlocks, x);
    note_launch(3);
    CU(cudaFreeAsync(red, s));
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_net_target(int nx, int ny, int nz, const double* u, float* t, void* stream) {
    if (!u || !t) return fail(GMG_ERR_ARG, "null argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(GMG_ERR_ARG, "grid must be at least 1 x 1 x 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = 3LL * (nx + 1) * (ny + 1) * (nz + 1);
    double* red = nullptr;
    CU(cudaMallocAsync(&red, sizeof(double) * (kRedBlocks + 1), s));
    k_reduce_vec<<<kRedBlocks, kRedThreads, 0, s>>>(u, n, 1, red);
    k_finish_vec<<<1, 256, 0, s>>>(red, kRedBlocks, 1, red + kRedBlocks);
    k_target<<<blocks_for(n, 256), 256, 0, s>>>(u, n, red + kRedBlocks, t);
    note_launch(3);
    CU(cudaFreeAsync(red, s));
    CU(cudaGetLastError());
    return GMG_OK;
}

int gmg_warm_start(gmg_handle* h, gmg_net* net, const float* rho, const double* f, double* u0, double* alpha_out) {
    if (!h || !net || !rho || !f || !u0) return fail(GMG_ERR_ARG, "null argument");
    const gmg::Level& l0 = h->lev[0];
    TRY(check_dims(l0.nx, l0.ny, l0.nz, 1));
    cudaStream_t s = h->stream;
    const long long nn = l0.nn;
    if (net->ws_cap < nn) {
        for (void* p : {(void*)net->ws_g, (void*)net->ws_kg, (void*)net->ws_x}) {
            if (!p) continue;
            auto it = std::find(net->allocs.begin(), net->allocs.end(), p);
            if (it != net->allocs.end()) net->allocs.erase(it);
            cudaFree(p);
        }
        net->ws_g = net->ws_kg = net->ws_x = nullptr;
        net->ws_cap = 0;
        TRY(dalloc(net->allocs, &net->ws_g, 3 * nn));
        TRY(dalloc(net->allocs, &net->ws_kg, 3 * nn));
        TRY(dalloc(net->allocs, &net->ws_x, GMG_NET_IN * nn));
        net->ws_cap = nn;
    }
    Work* w = nullptr;
    TRY(get_work(net, l0.nx, l0.ny, l0.nz, 1, false, &w));
    // features (mask bits of the handle)
    k_load_stats<<<kRedBlocks, kRedThreads, 0, s>>>(f, nn, net->ws_red);
    k_load_stats_finish<<<1, 256, 0, s>>>(net->ws_red, kRedBlocks, net->ws_alpha + 1);
    k_features<<<blocks_for(nn, 256), 256, 0, s>>>(l0.nx, l0.ny, l0.nz, rho, f, nullptr, l0.mask, net->ws_alpha + 1,
                                                   net->ws_x);
    note_launch(3);
    TRY(forward(net, w, net->ws_x, w->g, 4, 4, s));
    k_out_to_dofs<<<blocks_for(3 * nn, 256), 256, 0, s>>>(w->g, l0.mask, nn, net->ws_g);
    note_launch();
    TRY(gmg_apply(h, net->ws_g, net->ws_kg));
    k_ws_dots<<<kRedBlocks, kRedThreads, 0, s>>>(f, net->ws_g, net->ws_kg, 3 * nn, net->ws_red);
    k_ws_alpha<<<1, 256, 0, s>>>(net->ws_red, kRedBlocks, net->ws_alpha);
    k_ws_scale<<<blocks_for(3 * nn, 256), 256, 0, s>>>(net->ws_g, 3 * nn, net->ws_alpha, u0);
    note_launch(3);
    CU(cudaGetLastError());
    if (alpha_out) {
        CU(cudaMemcpyAsync(alpha_out, net->ws_alpha, sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return GMG_OK;
}

void gmg_net_destroy(gmg_net* net) {
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    else cudaDeviceSynchronize();
    for (Work* w : net->works) {
        if (w->exec) cudaGraphExecDestroy(w->exec);
        if (w->exec_energy) cudaGraphExecDestroy(w->exec_energy);
        free_all(w->allocs);
        delete w;
    }
    if (net->cap) cudaStreamDestroy(net->cap);
    free_all(net->allocs);
    delete net;
}

}  // extern "C"
