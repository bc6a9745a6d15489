// Set-up kernels of the GMG hierarchy (sm_103a), all in FP64:
//
//  * SIMP moduli (Eq. simp_filter) and the unit hex8 stiffness K_e (Eq. state_eq),
//    integrated with the 2x2x2 Gauss rule from the tensor form
//    lambda dN_a/dx_c dN_b/dx_d + mu dN_a/dx_d dN_b/dx_c + mu delta_cd grad N_a . grad N_b;
//  * Dirichlet masks and their inheritance by injection (Sec. "Transfer
//    Operators and Boundary Masking");
//  * the level-1 Galerkin operator by local aggregation over the child
//    prolongation patterns (Eq. galerkin_level1), deeper levels by the
//    structured triple product R K P ("Coarser levels");
//  * diagonals, smoother coefficients (Algorithm cheb in the standard
//    Chebyshev semi-iteration form), the power-iteration finish
//    (Sec. "Spectral-radius estimation");
//  * the coarsest dense matrix with eps = max(mean_diag 1e-8, 1e-14), its
//    blocked right-looking Cholesky factor and the inverse (K^L + eps I)^{-1}.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace gmg {

namespace {

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

__global__ void k_moduli(const float* rho, long long ne, double p, double E0, double Emin, double* E64, float* E32) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        const double r = (double)rho[e];
        const double E = Emin + (E0 - Emin) * pow(r, p);
        E64[e] = E;
        E32[e] = (float)E;
    }
}

// dN_a/dx_k at xi in [0,1]^3 for the trilinear shape functions.
__device__ __forceinline__ void shape_grad(int a, double x, double y, double z, double g[3]) {
    const double fx = ldx(a) ? x : 1.0 - x, fy = ldy(a) ? y : 1.0 - y, fz = ldz(a) ? z : 1.0 - z;
    const double sx = ldx(a) ? 1.0 : -1.0, sy = ldy(a) ? 1.0 : -1.0, sz = ldz(a) ? 1.0 : -1.0;
    g[0] = sx * fy * fz;
    g[1] = fx * sy * fz;
    g[2] = fx * fy * sz;
}

__global__ void k_element_stiffness(double nu, double* Ke) {
    const int I = threadIdx.x;  // 576 threads
    if (I >= 576) return;
    const int row = I / 24, col = I % 24;
    const int a = row / 3, c = row % 3, b = col / 3, d = col % 3;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    const double h = 0.5 / sqrt(3.0);
    const double pts[2] = {0.5 - h, 0.5 + h};
    double s = 0.0;
    for (int qz = 0; qz < 2; ++qz)
        for (int qy = 0; qy < 2; ++qy)
            for (int qx = 0; qx < 2; ++qx) {
                double ga[3], gb[3];
                shape_grad(a, pts[qx], pts[qy], pts[qz], ga);
                shape_grad(b, pts[qx], pts[qy], pts[qz], gb);
                double v = lam * ga[c] * gb[d] + mu * ga[d] * gb[c];
                if (c == d) v += mu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
                s += 0.125 * v;
            }
    Ke[I] = s;
}

__global__ void k_mask_clamp(uint8_t* mask, int nx, int ny, int nz) {
    const long long NX = nx + 1, nn = NX * (ny + 1) * (nz + 1);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x)
        mask[n] = (n % NX == 0) ? 7 : 0;
}

__global__ void k_mask_from_dofs(const uint8_t* fixed, uint8_t* mask, long long nn) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x)
        mask[n] = (uint8_t)((fixed[3 * n] ? 1 : 0) | (fixed[3 * n + 1] ? 2 : 0) | (fixed[3 * n + 2] ? 4 : 0));
}

__global__ void k_mask_inject(const uint8_t* fmask, int fnx, int fny, uint8_t* cmask, int cnx, int cny, int cnz) {
    const long long CX = cnx + 1, CY = cny + 1, nn = CX * CY * (cnz + 1);
    const long long FX = fnx + 1, FY = fny + 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const long long I = n % CX, J = (n / CX) % CY, K = n / (CX * CY);
        cmask[n] = fmask[2 * I + FX * (2 * J + FY * 2 * K)];
    }
}

__global__ void k_count_free(const uint8_t* mask, long long nn, int* out) {
    int cnt = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const uint8_t m = mask[n];
        cnt += !fixed_bit(m, 0) + !fixed_bit(m, 1) + !fixed_bit(m, 2);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// 1D local prolongation weights W[pattern][fine local node][coarse local node]:
// pattern 0 = first child (fine nodes 2C, 2C+1), 1 = second child (2C+1, 2C+2),
// 2 = the clamped last child of an odd count (2nc, 2nc+1 -> coarse node nc).
__device__ __forceinline__ double w1(int pat, int f, int c) {
    if (pat == 0) return f == 0 ? (c == 0 ? 1.0 : 0.0) : 0.5;
    if (pat == 1) return f == 1 ? (c == 1 ? 1.0 : 0.0) : 0.5;
    return c == 1 ? 1.0 : 0.0;
}

__device__ __forceinline__ double w3(int pat, int a, int b) {
    return w1(pat % 3, ldx(a), ldx(b)) * w1((pat / 3) % 3, ldy(a), ldy(b)) * w1(pat / 9, ldz(a), ldz(b));
}

// M[pat] = P_pat^T K_e P_pat on the coarse element's 24 DOFs, for the 27 patterns.
__global__ void k_child_patterns(const double* Ke, double* M) {
    const int pat = blockIdx.x;
    for (int e = threadIdx.x; e < 576; e += blockDim.x) {
        const int I = e / 24, J = e % 24;
        const int bi = I / 3, ci = I % 3, bj = J / 3, cj = J % 3;
        double s = 0.0;
        for (int a = 0; a < 8; ++a) {
            const double wa = w3(pat, a, bi);
            if (wa == 0.0) continue;
            for (int a2 = 0; a2 < 8; ++a2) {
                const double wb = w3(pat, a2, bj);
                if (wb == 0.0) continue;
                s += wa * Ke[(3 * a + ci) * 24 + 3 * a2 + cj] * wb;
            }
        }
        M[pat * 576 + e] = s;
    }
}

// Fine elements whose coarse parent along one axis is C, with their patterns.
__device__ __forceinline__ int children_1d(int C, int nf, int* e, int* pat) {
    const int nc = nf >> 1;
    int n = 0;
    e[n] = 2 * C; pat[n++] = 0;
    e[n] = 2 * C + 1; pat[n++] = 1;
    if ((nf & 1) && C == nc - 1) { e[n] = nf - 1; pat[n++] = 2; }
    return n;
}

// K_C = sum over the fine children c of coarse element C of E_c P_c^T K_e P_c,
// with the rows of P_c that belong to fixed fine DOFs removed (Eq. galerkin_level1).
// One block of 192 threads per coarse element; 3 entries per thread.
__global__ void __launch_bounds__(192) k_coarse_element_matrices(int fnx, int fny, int fnz, const double* E,
                                                                 const uint8_t* fmask, const double* Ke,
                                                                 const double* M, double* Kc) {
    const int cnx = fnx >> 1, cny = fny >> 1;
    const long long C = blockIdx.x;
    const int Cx = (int)(C % cnx), Cy = (int)((C / cnx) % cny), Cz = (int)(C / ((long long)cnx * cny));
    int ex[3], px[3], ey[3], py[3], ez[3], pz[3];
    const int sx = children_1d(Cx, fnx, ex, px), sy = children_1d(Cy, fny, ey, py), sz = children_1d(Cz, fnz, ez, pz);
    const long long FX = fnx + 1, FY = fny + 1;
    double acc[3] = {0.0, 0.0, 0.0};
    __shared__ uint8_t cm[8];
    for (int kz = 0; kz < sz; ++kz)
        for (int ky = 0; ky < sy; ++ky)
            for (int kx = 0; kx < sx; ++kx) {
                const long long e = ex[kx] + (long long)fnx * (ey[ky] + (long long)fny * ez[kz]);
                const double Ee = E[e];
                const int pat = px[kx] + 3 * py[ky] + 9 * pz[kz];
                __syncthreads();
                if (threadIdx.x < 8) {
                    const int a = threadIdx.x;
                    cm[a] = fmask[(ex[kx] + ldx(a)) + FX * ((ey[ky] + ldy(a)) + FY * (ez[kz] + ldz(a)))];
                }
                __syncthreads();
                bool any = false;
                for (int a = 0; a < 8; ++a) any |= cm[a] != 0;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int idx = threadIdx.x + 192 * q;
                    if (!any) {
                        acc[q] += Ee * M[pat * 576 + idx];
                    } else {
                        const int I = idx / 24, J = idx % 24;
                        const int bi = I / 3, ci = I % 3, bj = J / 3, cj = J % 3;
                        double s = 0.0;
                        for (int a = 0; a < 8; ++a) {
                            if (fixed_bit(cm[a], ci)) continue;
                            const double wa = w3(pat, a, bi);
                            if (wa == 0.0) continue;
                            for (int a2 = 0; a2 < 8; ++a2) {
                                if (fixed_bit(cm[a2], cj)) continue;
                                const double wb = w3(pat, a2, bj);
                                if (wb == 0.0) continue;
                                s += wa * Ke[(3 * a + ci) * 24 + 3 * a2 + cj] * wb;
                            }
                        }
                        acc[q] += Ee * s;
                    }
                }
            }
#pragma unroll
    for (int q = 0; q < 3; ++q) Kc[C * 576 + threadIdx.x + 192 * q] = acc[q];
}

__global__ void k_fine_element_matrices(const double* E, long long ne, const double* Ke, double* Kc) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ne * 576; t += (long long)gridDim.x * blockDim.x)
        Kc[t] = E[t / 576] * Ke[t % 576];
}

// Owner-computes scatter of the coarse element matrices into the 27-slot planes
// of each coarse node (fixed order over elements: no atomics).
__global__ void k_gather_level1(int cnx, int cny, int cnz, long long nn, const double* Kc, double* A) {
    const long long CX = cnx + 1, CY = cny + 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(n % CX), J = (int)((n / CX) % CY), K = (int)(n / (CX * CY));
        for (int ea = 0; ea < 8; ++ea) {
            const int ox = I - ldx(ea), oy = J - ldy(ea), oz = K - ldz(ea);
            if (ox < 0 || ox >= cnx || oy < 0 || oy >= cny || oz < 0 || oz >= cnz) continue;
            const double* Ke = Kc + (ox + (long long)cnx * (oy + (long long)cny * oz)) * 576;
            for (int eb = 0; eb < 8; ++eb) {
                const int s = slot_of(ldx(eb) - ldx(ea), ldy(eb) - ldy(ea), ldz(eb) - ldz(ea));
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        A[(long long)(s * 9 + r * 3 + c) * nn + n] += Ke[(3 * ea + r) * 24 + 3 * eb + c];
            }
        }
    }
}

// Per-axis fine support of coarse node I with weights (Eq. trilinear_weights).
__device__ __forceinline__ int fine_support64(int I, int nf, int* idx, double* w) {
    const int nc = nf >> 1;
    int n = 0;
    idx[n] = 2 * I; w[n++] = 1.0;
    if (I >= 1) { idx[n] = 2 * I - 1; w[n++] = 0.5; }
    const int f = 2 * I + 1;
    if (f <= nf) { idx[n] = f; w[n++] = (f < 2 * nc) ? 0.5 : 1.0; }
    return n;
}

// Pairs (fine i in supp(I), fine j in supp(J)) with |i - j| <= 1 along one axis.
__device__ __forceinline__ int axis_pairs(int I, int Jc, int nf, int* fi, int* df, double* w) {
    int si[3], sj[3];
    double wi[3], wj[3];
    const int ni = fine_support64(I, nf, si, wi), nj = fine_support64(Jc, nf, sj, wj);
    int n = 0;
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < nj; ++b) {
            const int d = sj[b] - si[a];
            if (d >= -1 && d <= 1) { fi[n] = si[a]; df[n] = d; w[n] = wi[a] * wj[b]; ++n; }
        }
    return n;
}

// K^{l+1}(N, N+o) = sum_{i in supp N} sum_{j in supp(N+o)} w_i w_j K^l(i, j) for the
// 27-point fine operator (structured Galerkin triple product).  One thread per
// (coarse node, slot).
__global__ void k_galerkin_rap(int fnx, int fny, int fnz, long long fnn, const double* Af, int cnx, int cny, int cnz,
                               long long cnn, double* Ac) {
    const long long total = cnn * kSlots;
    const long long CX = cnx + 1, CY = cny + 1, CZ = cnz + 1;
    const long long FX = fnx + 1, FY = fny + 1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long n = t % cnn;
        const int s = (int)(t / cnn);
        const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = s / 9 - 1;
        const int I = (int)(n % CX), J = (int)((n / CX) % CY), K = (int)(n / (CX * CY));
        const int MI = I + ox, MJ = J + oy, MK = K + oz;
        double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (MI >= 0 && MI < CX && MJ >= 0 && MJ < CY && MK >= 0 && MK < CZ) {
            int fx[9], dx[9], fy[9], dy[9], fz[9], dz[9];
            double wx[9], wy[9], wz[9];
            const int nx_ = axis_pairs(I, MI, fnx, fx, dx, wx);
            const int ny_ = axis_pairs(J, MJ, fny, fy, dy, wy);
            const int nz_ = axis_pairs(K, MK, fnz, fz, dz, wz);
            for (int c = 0; c < nz_; ++c)
                for (int b = 0; b < ny_; ++b)
                    for (int a = 0; a < nx_; ++a) {
                        const double w = wx[a] * wy[b] * wz[c];
                        const long long fi = fx[a] + FX * (fy[b] + FY * fz[c]);
                        const int fs = slot_of(dx[a], dy[b], dz[c]);
                        const double* src = Af + (long long)(fs * 9) * fnn + fi;
#pragma unroll
                        for (int e = 0; e < 9; ++e) blk[e] = fma(w, src[(long long)e * fnn], blk[e]);
                    }
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) Ac[(long long)(s * 9 + e) * cnn + n] = blk[e];
    }
}

// Zero rows/columns of fixed DOFs and out-of-grid neighbours, form D^{-1} from
// the self block, and write the FP32 copy used by the solve: the diagonal block
// and the 13 forward neighbour blocks (slots 13..26) of the symmetric operator.
__global__ void k_finish_bsr(int nx, int ny, int nz, long long nn, long long ps, const uint8_t* mask, double* A64,
                             float* A32, float* invdiag) {
    const long long NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / (NX * NY));
        const uint8_t mr = mask[n];
        for (int s = 0; s < kSlots; ++s) {
            const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = s / 9 - 1;
            const bool in = i + ox >= 0 && i + ox < NX && j + oy >= 0 && j + oy < NY && k + oz >= 0 && k + oz < NZ;
            const uint8_t mc = in ? mask[n + ox + NX * (oy + NY * oz)] : 7;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const long long q = (long long)(s * 9 + r * 3 + c) * nn + n;
                    double v = A64[q];
                    if (!in || fixed_bit(mr, r) || fixed_bit(mc, c)) v = 0.0;
                    A64[q] = v;
                    if (s >= kSelfSlot) A32[(long long)((s - kSelfSlot) * 9 + r * 3 + c) * ps + n] = (float)v;
                }
        }
        for (int r = 0; r < 3; ++r) {
            const double dg = A64[(long long)(kSelfSlot * 9 + r * 3 + r) * nn + n];
            invdiag[3 * n + r] = fixed_bit(mr, r) ? 0.f : (float)(1.0 / dg);
        }
    }
}

// Per-step smoother coefficients (c_d, c_a): x_{k+1} = x_k + d_k,
// d_k = c_d d_{k-1} + c_a D^{-1} (b - K x_k).
//   Jacobi:    c_d = 0, c_a = omega.
//   Chebyshev: band [alpha lam, lam], lam = safety * estimate, theta = (1+alpha) lam / 2,
//              delta = (1-alpha) lam / 2, s = theta/delta, rho_0 = 1/s;
//              step 0: (0, 1/theta); step k: rho_k = 1/(2 s - rho_{k-1}),
//              (rho_k rho_{k-1}, 2 rho_k / delta).
__global__ void k_smoother_coef(double* coef, const double* lam_p, int kind, int degree, double omega, double alpha,
                                double safety) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (kind == GMG_SMOOTHER_JACOBI) {
        for (int k = 0; k < degree; ++k) { coef[2 * k] = 0.0; coef[2 * k + 1] = omega; }
        return;
    }
    const double lam = safety * lam_p[0];
    const double theta = 0.5 * (1.0 + alpha) * lam, delta = 0.5 * (1.0 - alpha) * lam;
    const double s1 = theta / delta;
    double rho = 1.0 / s1;
    coef[0] = 0.0;
    coef[1] = 1.0 / theta;
    for (int k = 1; k < degree; ++k) {
        const double rn = 1.0 / (2.0 * s1 - rho);
        coef[2 * k] = rn * rho;
        coef[2 * k + 1] = 2.0 * rn / delta;
        rho = rn;
    }
}

__global__ void k_lambda_finish(double* sc, double* lam_slot) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double floor_ = 1e-6;
    double lam = sc[SC_VKV] / sc[SC_VDV];
    if (sc[SC_TMP] != 0.0 || !isfinite(lam) || !(lam > floor_)) lam = floor_;
    lam_slot[0] = lam;
}

__global__ void k_free_index(const uint8_t* mask, long long nn, int* free_idx, int* count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 0;
    for (long long q = 0; q < 3 * nn; ++q)
        if (!fixed_bit(mask[q / 3], (int)(q % 3))) {
            if (free_idx) free_idx[c] = (int)q;
            ++c;
        }
    *count = c;
}

__global__ void k_dense_gather(int nx, int ny, long long nn, const double* A, const int* free_idx, int n, double* dense) {
    const long long NX = nx + 1, NY = ny + 1;
    const long long total = (long long)n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / n), b = (int)(t % n);
        const int fa = free_idx[a], fb = free_idx[b];
        const long long na = fa / 3, nb = fb / 3;
        const int r = fa % 3, c = fb % 3;
        const int ox = (int)(nb % NX - na % NX), oy = (int)((nb / NX) % NY - (na / NX) % NY),
                  oz = (int)(nb / (NX * NY) - na / (NX * NY));
        double v = 0.0;
        if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1)
            v = A[(long long)(slot_of(ox, oy, oz) * 9 + r * 3 + c) * nn + na];
        dense[t] = v;
    }
}

__global__ void k_regularise(double* A, int n, double* eps_out) {
    __shared__ double part[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += A[(long long)i * n + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    const double eps = fmax(part[0] / n * 1e-8, 1e-14);
    for (int i = threadIdx.x; i < n; i += 256) A[(long long)i * n + i] += eps;
    if (threadIdx.x == 0) *eps_out = eps;
}

constexpr int NB = 32;

// Unblocked Cholesky of the kb x kb diagonal block at (k0, k0) (row-major, lower).
__global__ void k_potrf_diag(double* A, int n, int k0, int kb, int* info) {
    __shared__ double s[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;  // (32, 32)
    if (tx < kb && ty < kb) s[ty][tx] = A[(long long)(k0 + ty) * n + k0 + tx];
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (tx == 0 && ty == 0) {
            const double d = s[j][j];
            if (!(d > 0.0) || !isfinite(d)) { *info = k0 + j + 1; s[j][j] = 1.0; }
            else s[j][j] = sqrt(d);
        }
        __syncthreads();
        if (tx == 0 && ty > j && ty < kb) s[ty][j] /= s[j][j];
        __syncthreads();
        if (ty > j && ty < kb && tx > j && tx <= ty) s[ty][tx] -= s[ty][j] * s[tx][j];
        __syncthreads();
    }
    if (tx < kb && ty < kb && tx <= ty) A[(long long)(k0 + ty) * n + k0 + tx] = s[ty][tx];
}

// Rows i >= k0+kb of the panel: L_ik = A_ik L_kk^{-T} (forward substitution per row).
__global__ void k_trsm_panel(double* A, int n, int k0, int kb) {
    __shared__ double Lk[NB][NB + 1];
    for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) Lk[t / kb][t % kb] = A[(long long)(k0 + t / kb) * n + k0 + t % kb];
    __syncthreads();
    const int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[NB];
    for (int j = 0; j < kb; ++j) {
        double v = A[(long long)i * n + k0 + j];
        for (int m = 0; m < j; ++m) v -= x[m] * Lk[j][m];
        x[j] = v / Lk[j][j];
    }
    for (int j = 0; j < kb; ++j) A[(long long)i * n + k0 + j] = x[j];
}

// Trailing update A_ij -= sum_m L_im L_jm for i >= j >= k0+kb (lower triangle).
__global__ void k_syrk(double* A, int n, int k0, int kb) {
    const int t0 = k0 + kb;
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    __shared__ double Li[NB][NB + 1], Lj[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = t0 + bi * NB + ty, j = t0 + bj * NB + tx;
    const int ri = t0 + bi * NB + ty, rj = t0 + bj * NB + ty;
    Li[ty][tx] = (ri < n && tx < kb) ? A[(long long)ri * n + k0 + tx] : 0.0;
    Lj[ty][tx] = (rj < n && tx < kb) ? A[(long long)rj * n + k0 + tx] : 0.0;
    __syncthreads();
    if (i < n && j < n && j <= i) {
        double s = 0.0;
        for (int m = 0; m < kb; ++m) s += Li[ty][m] * Lj[tx][m];
        A[(long long)i * n + j] -= s;
    }
}

// Column j of X = L^{-1} (lower triangular), by forward substitution.
__global__ void k_trinv_col(const double* L, int n, double* X) {
    extern __shared__ double x[];
    __shared__ double red[256];
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += 256) x[i] = 0.0;
    __syncthreads();
    for (int i = j; i < n; ++i) {
        double s = 0.0;
        for (int m = j + threadIdx.x; m < i; m += 256) s += L[(long long)i * n + m] * x[m];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) x[i] = ((i == j ? 1.0 : 0.0) - red[0]) / L[(long long)i * n + i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += 256) X[(long long)i * n + j] = x[i];
}

// Ainv = X^T X with X lower triangular: Ainv_ij = sum_{m >= max(i,j)} X_mi X_mj.
__global__ void k_xtx(const double* X, int n, double* Ainv) {
    __shared__ double Xi[NB][NB + 1], Xj[NB][NB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * NB + ty, j = blockIdx.x * NB + tx;
    const int m0 = max(blockIdx.y, blockIdx.x) * NB;
    double s = 0.0;
    for (int mb = m0; mb < n; mb += NB) {
        const int m = mb + ty;
        Xi[ty][tx] = (m < n && blockIdx.y * NB + tx < n) ? X[(long long)m * n + blockIdx.y * NB + tx] : 0.0;
        Xj[ty][tx] = (m < n && blockIdx.x * NB + tx < n) ? X[(long long)m * n + blockIdx.x * NB + tx] : 0.0;
        __syncthreads();
        for (int q = 0; q < NB; ++q) s += Xi[q][ty] * Xj[q][tx];
        __syncthreads();
    }
    if (i < n && j < n) Ainv[(long long)i * n + j] = s;
}

// The level-0 mask in the vectors' numbering (rows of px nodes; pad nodes fixed).
__global__ void k_mask_pad(const uint8_t* mask, int NX, int px, long long nnp, uint8_t* maskp) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnp; q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / px;
        const int i = (int)(q - row * px);
        maskp[q] = i < NX ? mask[row * NX + i] : (uint8_t)7;
    }
}

// DOF indices in the dense numbering -> the same DOFs in the level-0 vectors' numbering.
__global__ void k_pad_index(const int* idx, int n, int NX, int px, int* out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int dof = idx[q], node = dof / 3;
        out[q] = 3 * (node + (node / NX) * (px - NX)) + dof % 3;
    }
}

}  // namespace

static int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148 * 8)); }

void launch_moduli(const float* rho, long long ne, double p, double E0, double Emin, double* E64, float* E32,
                   cudaStream_t s) {
    note_launch();
    k_moduli<<<grid_for(ne), 256, 0, s>>>(rho, ne, p, E0, Emin, E64, E32);
}

void launch_element_stiffness(double nu, double* Ke, cudaStream_t s) {
    note_launch();
    k_element_stiffness<<<1, 576, 0, s>>>(nu, Ke);
}

void launch_mask_clamp(uint8_t* mask, int nx, int ny, int nz, cudaStream_t s) {
    const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    note_launch();
    k_mask_clamp<<<grid_for(nn), 256, 0, s>>>(mask, nx, ny, nz);
}

void launch_mask_from_dofs(const uint8_t* fixed_dofs, uint8_t* mask, long long nn, cudaStream_t s) {
    note_launch();
    k_mask_from_dofs<<<grid_for(nn), 256, 0, s>>>(fixed_dofs, mask, nn);
}

void launch_mask_inject(const Level& f, Level& c, cudaStream_t s) {
    note_launch();
    k_mask_inject<<<grid_for(c.nn), 256, 0, s>>>(f.mask, f.nx, f.ny, c.mask, c.nx, c.ny, c.nz);
}

void launch_mask_pad(const Level& l0, cudaStream_t s) {
    note_launch();
    k_mask_pad<<<grid_for(l0.nnp), 256, 0, s>>>(l0.mask, l0.nx + 1, l0.px, l0.nnp, l0.maskp);
}

void launch_pad_index(const int* idx, int n, const Level& l0, int* out, cudaStream_t s) {
    note_launch();
    k_pad_index<<<grid_for(n), 256, 0, s>>>(idx, n, l0.nx + 1, l0.px, out);
}

void launch_count_free(const uint8_t* mask, long long nn, int* out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, sizeof(int), s);
    note_launch();
    k_count_free<<<grid_for(nn), 256, 0, s>>>(mask, nn, out);
}

void launch_child_patterns(const double* Ke, double* Mpat, cudaStream_t s) {
    note_launch();
    k_child_patterns<<<27, 192, 0, s>>>(Ke, Mpat);
}

void launch_coarse_element_matrices(int nx, int ny, int nz, const double* E, const uint8_t* fine_mask, const double* Ke,
                                    const double* Mpat, double* Kc, cudaStream_t s) {
    const long long nce = (long long)(nx >> 1) * (ny >> 1) * (nz >> 1);
    if (nce > 0) { note_launch(); k_coarse_element_matrices<<<(unsigned)nce, 192, 0, s>>>(nx, ny, nz, E, fine_mask, Ke, Mpat, Kc); }
}

void launch_fine_element_matrices(const double* E, long long ne, const double* Ke, double* Kc, cudaStream_t s) {
    note_launch();
    k_fine_element_matrices<<<grid_for(ne * 576), 256, 0, s>>>(E, ne, Ke, Kc);
}

void launch_gather_level1(const Level& c, const double* Kc, double* A64, cudaStream_t s) {
    cudaMemsetAsync(A64, 0, sizeof(double) * kPlanes * c.nn, s);
    note_launch();
    k_gather_level1<<<grid_for(c.nn), 256, 0, s>>>(c.nx, c.ny, c.nz, c.nn, Kc, A64);
}

void launch_galerkin_rap(const Level& f, const Level& c, cudaStream_t s) {
    note_launch();
    k_galerkin_rap<<<grid_for(c.nn * kSlots), 256, 0, s>>>(f.nx, f.ny, f.nz, f.nn, f.A64, c.nx, c.ny, c.nz, c.nn, c.A64);
}

void launch_finish_bsr(Level& l, cudaStream_t s) {
    note_launch();
    k_finish_bsr<<<grid_for(l.nn), 256, 0, s>>>(l.nx, l.ny, l.nz, l.nn, l.ps, l.mask, l.A64, l.A32, l.invdiag);
}

void launch_smoother_coef(double* coef, const double* lam, int kind, int degree, double omega, double alpha,
                          double safety, cudaStream_t s) {
    note_launch();
    k_smoother_coef<<<1, 32, 0, s>>>(coef, lam, kind, degree, omega, alpha, safety);
}

void launch_lambda_finish(double* sc, double* lam_slot, cudaStream_t s) {
    note_launch();
    k_lambda_finish<<<1, 32, 0, s>>>(sc, lam_slot);
}

void launch_free_index(const uint8_t* mask, long long nn, int* free_idx, int* count, cudaStream_t s) {
    note_launch();
    k_free_index<<<1, 32, 0, s>>>(mask, nn, free_idx, count);
}

void launch_dense_gather(const Level& l, const int* free_idx, int n, double* dense, cudaStream_t s) {
    note_launch();
    k_dense_gather<<<grid_for((long long)n * n), 256, 0, s>>>(l.nx, l.ny, l.nn, l.A64, free_idx, n, dense);
}

void launch_regularise(double* dense, int n, double* eps_out, cudaStream_t s) {
    note_launch();
    k_regularise<<<1, 256, 0, s>>>(dense, n, eps_out);
}

// Factor A (n x n, row-major, in place, lower triangle) and write (A)^{-1} to Ainv.
// work: n*n doubles.  Returns GMG_OK, GMG_ERR_CHOLESKY or GMG_ERR_CUDA.
int cholesky_and_inverse(double* A, int n, double* work, int* info_dev, double* Ainv, cudaStream_t s) {
    if (n <= 0) return GMG_OK;
    cudaMemsetAsync(info_dev, 0, sizeof(int), s);
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int kb = std::min(NB, n - k0);
        note_launch();
        k_potrf_diag<<<1, dim3(NB, NB), 0, s>>>(A, n, k0, kb, info_dev);
        const int rest = n - k0 - kb;
        if (rest > 0) {
            note_launch();
            k_trsm_panel<<<(rest + 127) / 128, 128, 0, s>>>(A, n, k0, kb);
            const int nbt = (rest + NB - 1) / NB;
            note_launch();
            k_syrk<<<dim3(nbt, nbt), dim3(NB, NB), 0, s>>>(A, n, k0, kb);
        }
    }
    int info = 0;
    if (cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GMG_ERR_CUDA;
    if (info != 0) return GMG_ERR_CHOLESKY;
    const size_t shm = sizeof(double) * (size_t)n;
    if (shm > 48 * 1024) cudaFuncSetAttribute(k_trinv_col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    note_launch();
    k_trinv_col<<<n, 256, shm, s>>>(A, n, work);
    const int nbt = (n + NB - 1) / NB;
    note_launch();
    k_xtx<<<dim3(nbt, nbt), dim3(NB, NB), 0, s>>>(work, n, Ainv);
    if (cudaGetLastError() != cudaSuccess) return GMG_ERR_CUDA;
    return GMG_OK;
}

}  // namespace gmg
